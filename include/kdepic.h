/*
 * kdepic.h -- C ABI of the GB300 (sm_103a) KDE particle-in-cell hot path.
 *
 * Method: Wu & Qin, "Reducing Noise for PIC Simulations Using Kernel Density
 * Estimation Algorithm" (arXiv 1804.11174).  The library deposits particle
 * charge on a 1D periodic grid with von Mises shape functions (Sec. II.A,
 * Eq. vonMises; Eq. kde), gathers the field back through the same kernels,
 * selects widths by leave-one-out cross-validation (Sec. II.B, Eq. cv_def),
 * adapts them per particle (Sec. II.C) and advances an electrostatic
 * leap-frog PIC cycle (Sec. III.A).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Domain x in [0, L) is periodic; theta = 2 pi x / L.  Positions are passed
 *   as 32-bit periodic fixed-point codes u = floor(x / L * 2^32) (uint32).
 *   Grid node g sits at x_g = g L / Ng.
 * - Kernel: K_kappa(theta) = exp(kappa (cos theta - 1)) / (2 pi I0e(kappa)),
 *   I0e(kappa) = exp(-kappa) I0(kappa).  kappa must be finite, in (0, 1e6].
 * - Pointers: every array argument is a DEVICE pointer unless its comment says
 *   "host".  The caller owns every buffer; the library never frees or keeps a
 *   caller pointer past the call (pic_step updates the caller's state arrays
 *   in place).  The context owns only its internal workspace.
 * - Precision: arrays documented as `real` are float32 by default and float64
 *   when the call's flags include KDE_F64.  Positions are always uint32.
 * - Ordering: calls enqueue work on the context's stream and return without
 *   synchronising, except those that return host values (kde_cv, kde_sync).
 *   A context's calls must not overlap on the GPU (they share its workspace
 *   and scratch words): use one context per stream or host thread.
 * - Errors: every call returns a kde_status.  Arguments are validated on the
 *   host before anything is launched; on failure nothing is enqueued and
 *   kde_last_error() describes the problem.  Device-side problems (a width out
 *   of range, a wait that ran out of iterations) set a status word on the
 *   device that the next kde_sync() (or kde_cv) reports as KDE_EDEVICE.
 * - Workspace: the first call at a new problem size may grow the context's
 *   workspace with cudaMalloc.  kde_reserve() grows it up front (do that before
 *   capturing calls into a CUDA graph).
 * - Determinism: for fixed inputs and sizes every result is bitwise
 *   reproducible (fixed summation orders; the deposit combines per-chunk sums
 *   with integer atomics).
 */
#ifndef KDEPIC_H
#define KDEPIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kde_ctx kde_ctx;
typedef int kde_status;

#define KDE_OK 0
#define KDE_EINVAL 1   /* invalid argument (host-side validation) */
#define KDE_ENOMEM 2   /* workspace allocation failed */
#define KDE_ECUDA 3    /* a CUDA runtime call failed */
#define KDE_EDEVICE 4  /* a kernel reported a problem through the device status word */
#define KDE_ENOTSUP 5  /* combination of options not supported */
#define KDE_ECANCELED 6 /* request server: the request was cancelled before it started */
#define KDE_EBUSY 7     /* request server: the request has started and can no longer be cancelled */

/* flags */
#define KDE_F64 0x1u         /* real arrays are float64 and arithmetic is FP64 */
#define KDE_POISSON_FD 0x2u  /* finite-difference Poisson (Sec. III.A) instead of spectral */
#define KDE_CV_SCALE 0x4u    /* kde_cv: candidates scale per-particle widths kappa_rel */
#define KDE_CV_SPECTRAL 0x8u /* kde_cv / pic_step: exact Fourier form of the CV (uniform widths) */
#define KDE_CV_PAIRS 0x10u   /* kde_cv / pic_step: O(N^2) pair sums of the CV (uniform widths) */
/* Uniform candidate widths without either flag: both forms are exact, and a
 * cost rule picks the cheaper one per call -- the Fourier form when
 * 8 M(kappa_max) < N sum_c frac(kappa_c), with M(kappa) the Fourier modes the
 * exact form keeps and frac(kappa) the share of the circle inside a kernel's
 * truncation radius (pair sums cost N^2 frac / 2 exponentials per candidate,
 * the Fourier form about 4 N M(kappa_max) for all candidates together). */

/* Maximum grid size accepted by deposit / gather / Poisson / pic_step. */
#define KDE_MAX_NG 4096

/* Create a context bound to `device` and `stream` (a cudaStream_t; NULL selects
 * the legacy default stream).  *out receives the context; destroy it with
 * kde_destroy.  Returns KDE_ECUDA if the device cannot be used. */
kde_status kde_create(kde_ctx **out, int device, void *stream);

/* Release the context and its workspace (synchronises its stream first). */
kde_status kde_destroy(kde_ctx *ctx);

/* Rebind the context to another stream of the same device. */
kde_status kde_set_stream(kde_ctx *ctx, void *stream);

/* Human-readable description of the last failure on this context (never NULL). */
const char *kde_last_error(const kde_ctx *ctx);

/* Wait for the context's stream and report the device status word
 * (KDE_EDEVICE with a description if a kernel flagged a problem; the word is
 * cleared by this call). */
kde_status kde_sync(kde_ctx *ctx);

/* Autotuner (no counterpart in the paper: a speed facility of this library).  Keys are
 * (grid size, log2 N, uniform width to a quarter octave, or "per-particle widths").
 *  - Tile shape of the FP32 gather.  The packed gather has several tile shapes
 *    (particles a lane, node-loop unrolling, launch bound) that give bitwise-identical
 *    results.  The first FP32 gather (kde_gather, or the gather and push of pic_step
 *    and of the ensemble) of each key runs every shape twice on its own data, timed by
 *    CUDA events, and keeps the fastest for that key.
 *  - Truncation radius of the FP32 PIC step (see kde_set_truncation).  Unless a cut is
 *    fixed, the first FP32 pic_step of each key runs the deposit + field and a gather
 *    on the step's own sorted particles at the cuts 2^-24, 2^-20 and 2^-18 of each
 *    kernel's peak, in rounds timed by CUDA events; a cut is admitted when it changes
 *    the results (a narrower window somewhere) and the node field and the particle
 *    fields match those of 2^-24 within 2.5e-6 relative L2, and is chosen when it is at
 *    least 3% faster than the best admitted cut so far.  Later steps with the key use
 *    it in their deposit and gather alike.
 * Later calls with a tuned key use the stored choice.  Tuning synchronises the stream
 * once per new key and is skipped while the stream is being captured (and, for the
 * gather, when an output aliases an input).  Off by default.  kde_autotune_entries
 * reports how many gather keys have been tuned; kde_autotune_table lists every stored
 * choice: keys[i] (bits 0-15 grid size, 16-23 log2 N, 24-31 width class: 0 for
 * per-particle widths, else 4 log2(kappa) + 128), kinds[i] (0: gather tile shape,
 * values[i] its index; 1: truncation, values[i] the cut exponent c of 2^-c), at most
 * cap entries written, *n_out = the number stored. */
kde_status kde_set_autotune(kde_ctx *ctx, int32_t enable);
kde_status kde_autotune_entries(const kde_ctx *ctx, int32_t *n_out);
kde_status kde_autotune_table(const kde_ctx *ctx, int32_t cap, uint64_t *keys, int32_t *kinds, double *values,
                              int32_t *n_out);
/* Stores n autotuner choices in the layout kde_autotune_table reports (a tuning table saved
 * from an earlier run): later calls with those keys use them without tuning.  KDE_EINVAL, and
 * nothing stored, unless every entry is a gather tile shape 0-2 or a cut exponent 24, 20 or 18. */
kde_status kde_autotune_set(kde_ctx *ctx, int32_t n, const uint64_t *keys, const int32_t *kinds,
                            const double *values);

/* Truncation of the FP32 deposit and gather (Eq. kde, evaluated over a finite window;
 * no counterpart in the paper, whose sums run over all nodes).  Every FP32 deposit and
 * gather evaluates each particle's kernel at least over the nodes where its weight is
 * 2^-c of its peak or more, c = log2_cut.  The kernel mass left outside is at most
 * 3.6e-8 (c = 24, the default), 5.8e-7 (20), 2.3e-6 (18) and 9.2e-6 (16) of the total,
 * over all widths (worst near kappa = 6-9; von Mises tail integrals).  log2_cut = 0
 * returns to the default, with pic_step's cut chosen by the autotuner when it is on.
 * KDE_EINVAL unless log2_cut is 0 or in [16, 40].  FP64 paths always cut at 2^-64; the CV's
 * pair sums and kde_deposit_noalloc (which takes no context) keep 2^-24. */
kde_status kde_set_truncation(kde_ctx *ctx, double log2_cut);

/* Launch overlap (no counterpart in the paper: a speed facility of this library).
 * With enable != 0 (the default) the kernels of the FP32 step chain -- the sort's scan
 * and scatter, the deposit, the field kernel and the gather with push -- are launched
 * as programmatic dependents: each may begin its independent prologue (loading its own
 * particles, building node tables) while the kernel before it in the stream finishes,
 * and waits on the device for that kernel's results before it reads them or writes
 * anything.  Results are bitwise identical with the setting on or off.  Launches that
 * follow a profiling event or another stream's work are ordered as usual. */
kde_status kde_set_launch_overlap(kde_ctx *ctx, int32_t enable);

/* Limit of the bounded device-side waits (no counterpart in the paper: a
 * robustness facility of this library).  The CV kernels stage column tiles with
 * bulk copies and wait for each on an mbarrier; a wait that has not seen its copy
 * land after `polls` polls gives up: the kernel waits (with the default limit)
 * for every copy it still has in flight, sets the device status word and stops,
 * and the next kde_cv / kde_sync returns KDE_EDEVICE ("device wait timed out").
 * The context stays usable.  polls < 0 restores the default (2^26 polls);
 * polls = 0 makes every such wait give up at once (this exercises the error path
 * without a fault).  KDE_EINVAL above 2^32 - 1. */
kde_status kde_set_wait_limit(kde_ctx *ctx, int64_t polls);

/* Grow the workspace for problems of up to N particles, grids of up to Ng nodes
 * and up to n_cand CV candidates, so that later calls allocate nothing. */
kde_status kde_reserve(kde_ctx *ctx, int64_t N, int32_t Ng, int32_t n_cand);

/* Position encoding on the periodic domain (Sec. III.A, periodic boundary):
 *   u_i = floor(frac(x_i / L) * 2^32),  frac(t) = t - floor(t),
 * with x_i / L the correctly rounded FP64 quotient, so positions outside [0, L)
 * wrap.  A fraction that rounds up to 1 (a tiny negative x_i) gives 2^32 - 1; a
 * NaN position gives 0.  x: device float64[N]; u_out: device uint32[N].
 * N >= 0 (N = 0 enqueues nothing), L > 0; KDE_EINVAL otherwise. */
kde_status kde_pack_positions(kde_ctx *ctx, const double *x, int64_t N, double L, uint32_t *u_out);

/* Deposit (Eq. kde at the grid nodes; per-particle widths as in Sec. II.C):
 *   rho_g = sum_i w_i (2 pi / L) K_{kappa_i}(theta_g - theta_i),  g = 0..Ng-1.
 * u: uint32[N] positions in any order.  kappa: real[N] per-particle widths, or
 * NULL to use kappa_uniform for every particle.  weight: real[N] non-negative
 * particle weights, or NULL for w_i = L / N (mean density 1).  rho_out:
 * real[Ng].  Terms below 2^-24 of a kernel's peak may be skipped (truncated
 * support).  N >= 0 (N = 0 gives zeros), 1 <= Ng <= KDE_MAX_NG, L > 0.
 * Flags: KDE_F64.  In FP32 the per-particle normalisations come from a table of
 * I0e built in FP64 when the context is created (relative error below 5e-7), and
 * chunks whose widths are all at most 32 use the form 2^(K cos(theta_g - theta_i) - K),
 * K = kappa log2(e), whose exponent carries about K 2^-24 of rounding error. */
kde_status kde_deposit(kde_ctx *ctx, const uint32_t *u, const void *kappa, double kappa_uniform,
                       const void *weight, int64_t N, int32_t Ng, double L, void *rho_out,
                       uint32_t flags);

/* Allocation-free deposit.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory once they run -- code
 * recording work into CUDA graphs, hosts whose allocator policy forbids device
 * allocations after start-up, and real-time loops that may not block on the
 * driver's allocator.  It computes what kde_deposit computes (same arguments,
 * same flags, same result within FP32 rounding) but takes a cudaStream_t
 * instead of a context, never calls cudaMalloc or cudaFree, and keeps all of
 * its scratch in one file-scope device array of KDE_NOALLOC_SCRATCH_BYTES
 * (98,560 bytes) that every GPU which loads the library holds until the
 * process exits.  Limits: Ng <= KDE_NOALLOC_MAX_NG (4096); larger grids return
 * KDE_EINVAL.  Particles may come in any order; cell-sorted input runs fastest
 * (an unsorted chunk falls back to every node of the grid).  Every call looks up
 * the array's address on the current device (cudaGetSymbolAddress, checked); the
 * first call on a device may load the library's module there, so make that first
 * call before any stream capture.  All calls share the one array,
 * which keeps the previous call's contents (the accumulators are cleared at
 * the start of each call): calls that overlap on the GPU -- on different
 * streams or from different host threads -- race and must be serialised by the
 * caller.  Out-of-range widths are clamped to 1e6 without a device status
 * report (there is no context to hold one).  Returns KDE_EINVAL on bad
 * arguments and KDE_ECUDA if the CUDA runtime refuses a launch or copy. */
#define KDE_NOALLOC_MAX_NG 4096
#define KDE_NOALLOC_SCRATCH_BYTES 98560
kde_status kde_deposit_noalloc(void *stream, const uint32_t *u, const void *kappa, double kappa_uniform,
                               const void *weight, int64_t N, int32_t Ng, double L, void *rho_out,
                               uint32_t flags);

/* Poisson solve on the periodic grid for the total charge density
 *   rho_total_g = background + charge * rho_g :
 * spectral (default): E_m = rho_m / (i k_m), k_m = 2 pi m / L, E_0 = 0 and, for
 * even Ng, E_{Ng/2} = 0; KDE_POISSON_FD: the finite-difference scheme of
 * Sec. III.A, whose Fourier symbol replaces k_m by (2/dx) tan(pi m / Ng).
 * rho: real[Ng]; E_out: real[Ng] (must not alias rho).  Also writes the field
 * energy 1/2 sum_g E_g^2 dx to energy_out (device float64[1]) if not NULL.
 * Flags: KDE_F64, KDE_POISSON_FD. */
kde_status kde_poisson(kde_ctx *ctx, const void *rho, int32_t Ng, double L, double charge,
                       double background, void *E_out, double *energy_out, uint32_t flags);

/* Gather through the deposit's kernels:
 *   out_i = sum_g (2 pi / Ng) K_{kappa_i}(theta_g - theta_i) field_g.
 * u: uint32[N] (any order); kappa: real[N] or NULL (kappa_uniform); field:
 * real[Ng]; out: real[N] in the order of u.  Flags: KDE_F64. */
kde_status kde_gather(kde_ctx *ctx, const uint32_t *u, const void *kappa, double kappa_uniform,
                      int64_t N, const void *field, int32_t Ng, double L, void *out,
                      uint32_t flags);

/* Leave-one-out cross-validation over candidate widths (Sec. II.B, Eq. cv_def):
 *   CV(c) = int fhat_c^2 dx - (2 / (n (n-1))) sum_i sum_{j != i} K_{kappa_jc}(x_i - x_j),
 * in x units (the kernel in x units is (2 pi / L) K).  Widths for candidate c:
 * kappa_jc = cand[c] (uniform), or cand[c] * kappa_rel[j] with KDE_CV_SCALE.
 * u: uint32[N] (any order), N >= 2; kappa_rel: float32[N] (KDE_CV_SCALE only);
 * cand: HOST float64[n_cand], 1 <= n_cand <= 256, each kappa in (0, 1e6];
 * cv_out: HOST float64[n_cand]; argmin_out: HOST int32 (smallest index on exact
 * ties), may be NULL; loo_out: float32[N] or NULL -- the leave-one-out density
 * (2 pi/L)(1/(n-1)) sum_{j != i} K_{kappa_j*}(theta_i - theta_j) at the selected
 * candidate, in the order of u.  Pair sums run in FP32 with per-tile FP64
 * accumulation; the integral term is an exact trapezoid sum on a grid fine
 * enough for the narrowest candidate; the final combination is FP64.  Pairs
 * whose kernel value is below 2^-24 of the peak may be skipped.  Synchronises.
 * KDE_CV_SPECTRAL (uniform widths only) evaluates the same objective by the
 * identity K(t) = (1/2pi) sum_m A_m e^{imt}, A_m = I_m/I_0: with the structure
 * factor S_m = sum_j e^{i m theta_j} (exact integer phases, FP64 combination),
 * the pair sum is (1/2pi)(n^2 + 2 sum A_m |S_m|^2) - n K(0) and the integral
 * term (1/(2pi n^2))(n^2 + 2 sum A_m^2 |S_m|^2), modes cut where A_m < 1e-17;
 * cost O(N sqrt(kappa_max)) instead of O(N^2) per candidate.  The
 * leave-one-out densities come from the same series (FP64 sums); their relative
 * accuracy degrades only for particles whose own kernel dominates their pilot
 * density.  Flags: KDE_CV_SCALE, KDE_CV_SPECTRAL. */
kde_status kde_cv(kde_ctx *ctx, const uint32_t *u, const float *kappa_rel, int64_t N, double L,
                  const double *cand, int32_t n_cand, double *cv_out, int32_t *argmin_out,
                  float *loo_out, uint32_t flags);

/* Particle-wise widths (Sec. II.C, Silverman): with the pilot density at the
 * CV width kappa_star, f~_i = ((n-1) loo_i + K_{kappa*}(0)) / n (x units),
 * log g = mean_i log f~_i, lambda_i = (f~_i / g)^(-alpha) and
 * kappa_i = kappa_star / lambda_i^2, clamped to [kappa_min, kappa_max].
 * loo: float32[N] as returned by kde_cv; kappa_out: float32[N].  The log-mean
 * is reduced in FP64.  N >= 2. */
kde_status kde_adapt_widths(kde_ctx *ctx, const float *loo, int64_t N, double L, double kappa_star,
                            double alpha, double kappa_min, double kappa_max, float *kappa_out);

/* Standard-PIC particle shapes, for the comparison of Sec. IV (Fig.
 * compare_high_order: shape order, kernel width and the KDE method).  The shape of
 * degree `order` (1 = CIC, 2, 3 or 5) and width h (x units) is the centred
 * cardinal B-spline S(x) = (1/h) B_order(x/h), support (order + 1) h; h = dx = L/Ng
 * is the standard PIC shape.  Not the paper's method: its baselines.
 * kde_deposit_bspline: rho_out[g] = sum_i (L/N) S(x_g - x_i) (periodic, point values
 *   at the nodes, x units); FP32 out, summed exactly in int64 fixed point, so the
 *   result does not depend on the particle order.  u: device uint32[N], any order.
 * kde_gather_bspline: out[i] = sum_g field[g] (dx/h) B_order((x_g - x_i)/h).
 * Both need order in {1, 2, 3, 5}, 0 < (order + 1) h < L, Ng <= KDE_MAX_NG. */
kde_status kde_deposit_bspline(kde_ctx *ctx, const uint32_t *u, int64_t N, int32_t order, double h, int32_t Ng,
                               double L, float *rho_out);
kde_status kde_gather_bspline(kde_ctx *ctx, const uint32_t *u, int64_t N, int32_t order, double h,
                              const float *field, int32_t Ng, double L, float *out);
/* Eq. (cv_def) for the first-order (CIC) shape over candidate widths h_c (HOST
 * float64[n_cand], 0 < h_c < L/4, n_cand <= 64), in x units:
 *   CV(h) = (1/n^2) sum_{i,j} (1/h) B_3((x_i - x_j)/h) - 2/(n(n-1)) sum_{i != j} (1/h) B_1((x_i - x_j)/h)
 * (B_1 * B_1 = B_3 gives the integral term exactly).  cv_out: HOST float64[n_cand];
 * argmin_out: smallest index on ties.  Pair sums in FP32 per tile, FP64 above.
 * Synchronises. */
kde_status kde_cv_cic(kde_ctx *ctx, const uint32_t *u, int64_t N, double L, const double *h_cand, int32_t n_cand,
                      double *cv_out, int32_t *argmin_out);

/* Anderson-Darling test of the positions against the uniform distribution on
 * the domain (Sec. II.D, where it decides when the width is re-optimised).
 * u: device uint32[N] position codes in any order (not modified); each sample
 * is taken at its code cell's centre, F_i = (u_i + 1/2) / 2^32.  N >= KDE_AD_MIN_N.
 * a2_out: the statistic A^2 = -n - (1/n) sum_i (2i - 1)[ln F_(i) + ln(1 - F_(n+1-i))];
 * log_p_out: natural log of the p-value -- Marsaglia & Marsaglia (2004) for
 * A^2 <= 7 (finite-n corrected), the limiting tail C (A^2)^{-1/2} e^{-A^2}
 * beyond.  Both HOST, either may be NULL.  Synchronises.  The sum runs in
 * FP64 with FP32 in-bin logarithms: |error of A^2| <= about 2e-11 N. */
#define KDE_AD_MIN_N 8
kde_status kde_ad_test(kde_ctx *ctx, const uint32_t *u, int64_t N, double *a2_out, double *log_p_out);

/* State of one electrostatic PIC run (Sec. III.A).  The caller owns all arrays.
 * pic_step reorders particles (u, v, kappa and id move together) by cell. */
typedef struct pic_state {
    uint32_t *u;          /* device uint32[N] positions (in/out) */
    void *v;              /* device real[N] velocities v^{n-1/2} (in/out) */
    void *kappa;          /* device real[N] per-particle widths (in/out), or NULL for uniform */
    void *kappa_norm;     /* device real[N] scratch kept equal to 1/(2 pi I0e(kappa_i)) by the
                             library (FP32: from the context's table, within 5e-7);
                             required when kappa != NULL */
    uint32_t *id;         /* device uint32[N] particle labels moved with the particles, or NULL */
    int64_t N;            /* particles, >= 1 */
    int32_t Ng;           /* grid nodes, 1..KDE_MAX_NG */
    double L, dt;         /* domain length and time step */
    double qm;            /* charge-to-mass ratio of the particles (-1 for electrons) */
    double charge;        /* charge per unit weight of the particles (-1 for electrons) */
    double background;    /* uniform neutralising background density (ions), usually 1 */
    double kappa_uniform; /* width when kappa == NULL (updated by the width schedule) */
    int32_t width_every;  /* > 0: run CV + width update every `width_every` steps */
    const double *cand;   /* HOST float64[n_cand] uniform-width candidates for the schedule */
    int32_t n_cand;
    double alpha;         /* Silverman sensitivity (0 = keep the uniform CV width) */
    double kappa_min, kappa_max; /* clamp for particle-wise widths */
    double *energy;       /* device float64[steps] field energy per step (indexed by step), or NULL */
    double *kappa_star;   /* device float64[steps] CV width in force per step, or NULL */
    int64_t step;         /* step counter (in/out); step 0 gets a half velocity kick */
    uint32_t flags;       /* KDE_F64, KDE_POISSON_FD, KDE_CV_SPECTRAL or KDE_CV_PAIRS (form of the
                             schedule's CV; neither: the cost rule), PIC_NO_BACKSTEP */
    /* Width-update algorithm of Sec. II.D on the uniform width (kappa == NULL;
     * replaces width_every).  Every step, before the deposit: ln p of the
     * Anderson-Darling test of the positions; if p > 2 ad_threshold then
     * p_th = 2 ad_threshold, else if p < p_th / 2 the CV over cand picks a
     * target width and p_th = p; then h = adjust_rate h_target +
     * (1 - adjust_rate) h with h = kappa_uniform^{-1/2}.  The caller's
     * kappa_uniform holds until the first optimisation, which sets h = h_target.
     * Reads the p-value on the host: one synchronisation per step. */
    int32_t width_ad;     /* != 0: use this schedule */
    double ad_threshold;  /* significance threshold (the paper uses 0.01) */
    double adjust_rate;   /* smoothing rate (the paper uses 0.05) */
    double ad_log_pth;    /* state, in/out: ln p_th; >= 0 means not started */
    double h_target;      /* state, in/out: target h of the last optimisation; 0 = none yet */
    int64_t n_opt;        /* state, in/out: optimisations so far */
    double *ad_log_p;     /* device float64[steps] ln p-value per step (indexed by step), or NULL */
    /* Standard PIC instead of the KDE deposit/gather (the baseline of the ensemble
     * comparison in Sec. III.B): shape_order 1 (CIC), 2, 3 or 5 selects the B-spline
     * shape of that degree and width shape_h (x units; 0 = dx) for the deposit and the
     * gather; FP32, no width schedule; particles are not reordered.  0 = von Mises. */
    int32_t shape_order;
    double shape_h;
} pic_state;

#define PIC_NO_BACKSTEP 0x100u /* do not halve the first kick at step 0 */

/* Advance the run by n_steps leap-frog steps.  Each step: (width update when
 * width_every > 0 and step % width_every == 0, or the Sec. II.D schedule when
 * width_ad != 0), counting sort by cell, deposit, Poisson, field energy,
 * gather, push.  At step 0 the velocity kick is halved
 * (v^{1/2} = v^0 + (q/m) E^0 dt / 2) unless PIC_NO_BACKSTEP.
 * Stream-ordered; no host synchronisation except the width_ad schedule's one
 * read of the p-value (and of the CV argmin on optimisation steps) per step. */
kde_status pic_step(kde_ctx *ctx, pic_state *st, int32_t n_steps);

/* pic_step on a state held in HOST memory (no counterpart in the paper: the
 * end-to-end form of the call for callers whose particles live on the host).
 * The pointer fields of *st -- u, v, kappa, id, and the histories energy,
 * kappa_star, ad_log_p (indexed by step) -- are HOST arrays of the sizes
 * pic_step documents; kappa_norm is ignored (the library keeps the norms on the
 * device).  The call copies the state into device buffers owned by the context,
 * runs n_steps of pic_step there, copies the state and the n_steps new history
 * entries back into the same host arrays, updates st's scalar state (step, the
 * uniform width and the Sec. II.D schedule state) and synchronises.  Page-locked
 * host memory makes the copies direct DMA; pageable memory works, more slowly.
 * Errors as pic_step; device buffers grow like the workspace. */
kde_status pic_step_host(kde_ctx *ctx, pic_state *st, int32_t n_steps);

/* Damping rate (Sec. III.B) from a field-energy history on the HOST: half the
 * slope of ln W through the first two strict local maxima at steps >= 1.
 * energy: HOST float64[n]; gamma_out: HOST.  Returns KDE_EINVAL if fewer than
 * two maxima exist. */
kde_status kde_damping_rate(const double *energy, int64_t n, double dt, double *gamma_out);

/* ---------------------------------------------------------------------------
 * Ensembles: R independent realisations of the PIC cycle of pic_step (uniform
 * width per realisation, q/m = -1, charge -1, background 1, spectral Poisson,
 * FP32) advanced together, as the ensemble statistics of Sec. III (MISE of the
 * density, damping rates over many loads) need.  The realisations' particles
 * are concatenated in the caller's device arrays u (uint32 codes) and v
 * (float32), realisation r occupying N[r] consecutive slots in order.  The
 * realisations are dealt to up to 16 lanes, each with its own context and
 * stream, so that they run concurrently; kde_ensemble_run can capture one step
 * of the whole ensemble into a CUDA graph and replay it once per step.  Each
 * realisation's results are bitwise those of pic_step on the same state.  The
 * arrays are reordered by cell within each realisation.  The lanes' contexts take
 * the autotune setting (kde_set_autotune) of ctx at creation and tune their gathers
 * in the first, uncaptured step.  Not a passage of the paper: the paper runs its
 * ensembles one after another.
 * ------------------------------------------------------------------------- */
typedef struct kde_ensemble kde_ensemble;

/* N, Ng, kappa: HOST arrays of R entries (1 <= N[r] < 2^32, 1 <= Ng[r] <=
 * KDE_MAX_NG, 0 < kappa[r] <= 1e6); u, v: device arrays of sum(N) entries,
 * owned by the caller and kept by the ensemble until kde_ensemble_destroy. */
kde_status kde_ensemble_create(kde_ctx *ctx, kde_ensemble **out, int32_t R, const int64_t *N, const int32_t *Ng,
                               const double *kappa, double L, double dt, uint32_t *u, float *v);
/* New uniform widths (HOST, R entries); a captured step is captured again. */
kde_status kde_ensemble_set_widths(kde_ensemble *ens, const double *kappa);
/* Standard PIC for every realisation (pic_state.shape_order / shape_h: B-spline of
 * degree order in {1, 2, 3, 5}, width h, 0 = dx), or order 0 for the von Mises KDE
 * step; a captured step is captured again. */
kde_status kde_ensemble_set_shape(kde_ensemble *ens, int32_t order, double h);
/* Integrated squared error of each realisation's deposited density against
 * 1 + alpha cos(2 pi mode x / L) at the current positions (one sample of the
 * MISE of Sec. II.B): mise (device float64[R]) = dx sum_g (rho_g - truth_g)^2. */
kde_status kde_ensemble_mise(kde_ensemble *ens, double alpha, int32_t mode, double *mise);
/* Advance every realisation by n_steps leap-frog steps (the first step of the
 * ensemble's life gets pic_step's half kick).  energy: device float64[R * n_steps],
 * energy[r * n_steps + k] = field energy of realisation r at step k of this call,
 * or NULL.  use_graph != 0 replays one captured step (captured once per
 * (energy, n_steps) pair).  Stream-ordered after and before the context's stream. */
kde_status kde_ensemble_run(kde_ensemble *ens, int32_t n_steps, double *energy, int32_t use_graph);
kde_status kde_ensemble_destroy(kde_ensemble *ens);

/* Measurement support: throughput probes used to derive the roofline of the
 * pair kernels (not part of the method).  Each launches a dependency-free
 * stream of `iters` operations per thread on all SMs and writes the elapsed
 * device time in ms to *ms_out (synchronises). */
kde_status kde_probe_exp2(kde_ctx *ctx, int64_t iters, double *ms_out, int64_t *ops_out);
kde_status kde_probe_fma(kde_ctx *ctx, int64_t iters, double *ms_out, int64_t *ops_out);

/* ---------------------------------------------------------------------------
 * Request server (continuous batching).  Not a passage of the paper: it serves
 * the operations above -- deposit, gather, CV and short PIC runs -- to many
 * concurrent requests.  n_slots slots each own a context and a CUDA stream and
 * run on their own host thread; submitted requests wait in one FIFO queue and
 * the head request starts as soon as a slot is idle and its device footprint
 * (inputs, outputs, workspace; see the implementation) fits in what is left of
 * hbm_budget_bytes.  Requests that arrive while others run therefore start as
 * slots and memory free up, and their kernels overlap on the device.  All
 * request buffers are HOST memory owned by the caller and must stay valid until
 * kde_server_wait returns for that ticket.  Every result is bitwise the same
 * whether the request ran alone or beside others.
 * ------------------------------------------------------------------------- */
typedef struct kde_server kde_server;

#define KDE_REQ_DEPOSIT 1 /* out: float32[Ng] density (kde_deposit) */
#define KDE_REQ_GATHER 2  /* field: float32[Ng]; out: float32[N] (kde_gather) */
#define KDE_REQ_CV 3      /* cand: float64[n_cand]; out64: float64[n_cand] CV; out_argmin */
#define KDE_REQ_PIC 4     /* v: float32[N]; n_steps, dt; out64: float64[n_steps] field energy;
                             out: float32[N] final velocities or NULL */

typedef struct kde_request {
    int32_t kind;            /* KDE_REQ_* */
    int64_t N;               /* particles */
    int32_t Ng;              /* grid nodes (1..KDE_MAX_NG) */
    double L;                /* domain length */
    const uint32_t *u;       /* HOST positions [N] */
    const float *kappa;      /* HOST per-particle widths [N] (CV: kappa_rel), or NULL */
    double kappa_uniform;    /* width when kappa == NULL (CV: candidates are widths) */
    const float *v;          /* HOST velocities [N] (PIC) */
    const float *field;      /* HOST field [Ng] (GATHER) */
    const double *cand;      /* HOST candidates (CV) */
    int32_t n_cand;
    int32_t n_steps;         /* PIC steps */
    double dt;               /* PIC time step */
    float *out;              /* HOST float32 output (see kinds) */
    double *out64;           /* HOST float64 output (see kinds) */
    int32_t *out_argmin;     /* HOST (CV), or NULL */
    uint32_t flags;          /* extra kde_cv flags for CV requests (KDE_CV_SPECTRAL) */
} kde_request;

/* Start a server with n_slots (1..64) slots on `device` under an HBM budget. */
kde_status kde_server_create(kde_server **out, int device, int32_t n_slots, int64_t hbm_budget_bytes);
/* Queue a request (validated here; KDE_EINVAL for bad fields or a footprint
 * larger than the whole budget); *ticket identifies it. */
kde_status kde_server_submit(kde_server *srv, const kde_request *req, int64_t *ticket);
/* Wait for a ticket; returns the request's status and the times (ms) from
 * submission and from admission to completion.  Each ticket is waited once. */
kde_status kde_server_wait(kde_server *srv, int64_t ticket, double *latency_ms, double *service_ms);
/* Like kde_server_wait, with the times in times[4]: latency from submission and
 * service time from admission (host clock, ms), then the device-clock interval
 * of the request on its slot's stream -- from an event recorded before its first
 * copy to one recorded after its last -- in ms since the server was created (-1
 * when not available, e.g. for a cancelled request).  Intervals of requests
 * served by different slots that intersect show their work overlapping. */
kde_status kde_server_wait_times(kde_server *srv, int64_t ticket, double *times);
/* Like kde_server_wait_times (times may be null), and for a failed request the
 * library's error message, NUL-terminated and truncated to msg_cap bytes, in msg
 * (an empty string for a request that succeeded; msg may be null when msg_cap is 0). */
kde_status kde_server_wait_msg(kde_server *srv, int64_t ticket, double *times, char *msg, int32_t msg_cap);
/* Cancel a request that is still queued: it never runs and its wait returns
 * KDE_ECANCELED.  KDE_EBUSY once it has been admitted (running or done);
 * KDE_EINVAL for an unknown ticket. */
kde_status kde_server_cancel(kde_server *srv, int64_t ticket);
/* HBM accounting and counters (host snapshot): stats[0] committed device bytes
 * now (transient buffers of running requests + workspace held by the slots'
 * contexts), stats[1] the largest committed total seen at an admission,
 * stats[2] the budget, stats[3] requests served, stats[4] cancelled, stats[5]
 * queued, stats[6] workspaces released to admit a request, stats[7] workspace
 * held now.  A request is admitted only while the committed total plus its
 * buffers and its slot's workspace growth fits the budget (or when it is the only
 * one running), so stats[1] stays within the budget unless a request's actual
 * workspace outgrows its estimate. */
kde_status kde_server_stats(kde_server *srv, int64_t *stats);
/* Finish the queued requests, stop the slots and release everything. */
kde_status kde_server_destroy(kde_server *srv);

/* Measurement support: while enabled, the library records CUDA events on its
 * stream around the launches of selected kernels and counts every kernel it
 * launches.  kde_profile_enable(ctx, on) synchronises, clears the record and
 * switches recording on or off.  kde_profile_read(ctx, kernel, &ms, &n)
 * synchronises and returns the summed device time and launch count of one
 * kernel: 0 CV pair sums, 1 deposit, 2 gather(+push), 3 sort scatter,
 * 4 Poisson, 5 CV integral-term deposit, 6 CV leave-one-out, 7 spectral
 * structure factor, 8 Anderson-Darling terms; kernel = -1
 * returns the number of all kernel launches in *n. */
kde_status kde_profile_enable(kde_ctx *ctx, int on);
kde_status kde_profile_read(kde_ctx *ctx, int kernel, double *total_ms, int64_t *launches);

#ifdef __cplusplus
}
#endif

#endif /* KDEPIC_H */
