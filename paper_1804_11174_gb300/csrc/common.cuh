// common.cuh -- internal definitions shared by the translation units of libkdepic.
//
// Position code: u = floor(x / L * 2^32); theta / 2 = pi u / 2^32.  All pair
// kernels evaluate the von Mises kernel as
//     exp(kappa (cos d - 1)) = exp(-2 kappa sin^2(d/2)) = 2^(-(beta sin(d/2))^2),
//     beta = sqrt(2 kappa log2 e),
// with sin(d/2) from the angle-difference identity on per-point half-angle
// sines and cosines, so one pair costs a few FMAs and one exp2.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <map>
#include <string>
#include <algorithm>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/kdepic.h"

#define KDE_PI 3.14159265358979323846
#define KDE_TWO_PI 6.28318530717958647692
#define KDE_LOG2E 1.44269504088896340736
#define KDE_LN2 0.69314718055994530942

// A kernel term whose exponent 2 kappa sin^2(d/2) log2 e exceeds the cut is
// below 2^-cut of the kernel's peak and may be skipped: 2^-24 in FP32, 2^-64
// in FP64 (below the rounding of either precision).
#define KDE_XCUT 24.0
#define KDE_XCUT64 64.0
template <typename T> struct KdeCut { static constexpr double x = KDE_XCUT; };
template <> struct KdeCut<double> { static constexpr double x = KDE_XCUT64; };
#define KDE_KAPPA_MAX 1.0e6

// device status word codes (first failure wins)
#define KDE_DEV_KAPPA_RANGE 1u
#define KDE_DEV_WAIT_TIMEOUT 2u
#define KDE_DEV_BAD_ARG 3u

// workspace slots owned by a context
enum WsSlot {
    WS_SORT_COUNTS = 0,
    WS_SORT_STARTS,
    WS_SORT_U,
    WS_SORT_P0,
    WS_SORT_P1,
    WS_SORT_P2,
    WS_SORT_P3,
    WS_SORT_P1B,  // the PIC step's second set of sorted widths, norms and labels
    WS_SORT_P2B,
    WS_SORT_P3B,
    WS_SORT_PERM,
    WS_NORM,
    WS_ACC,
    WS_GRID0,
    WS_GRID1,
    WS_WMAX,
    WS_CV_SC,
    WS_CV_TILE,
    WS_CV_KR,
    WS_CV_LNORM,
    WS_CV_PART,
    WS_CV_F2,
    WS_CV_TOT,
    WS_CV_OUT,
    WS_CV_CAND,
    WS_CV_ACC,
    WS_CV_LOO,
    WS_CV_RED,
    WS_PIC_E,
    WS_PIC_LOO,
    WS_PIC_KS,
    WS_SP_PART,
    WS_SP_S,
    WS_SP_A,
    WS_SP_ASEL,
    WS_SP_AS,
    WS_SP_SEL,
    WS_SP_MLIM,
    WS_AD_Z,
    WS_AD_T,
    WS_AD_PART,
    WS_AD_OUT,
    WS_CV_GPAR,
    WS_GREEN,
    WS_DEP_ROWS,   // persistent FP32 deposit: per-CTA node rows and their headers
    WS_HOST_U,     // device copies of a host-resident PIC state (pic_step_host)
    WS_HOST_V,
    WS_HOST_K,
    WS_HOST_NORM,
    WS_HOST_ID,
    WS_HOST_HIST,  // energy, kappa* and ln p histories
    WS_TUNE,       // truncation tuner: reference and candidate fields and their error sums
    WS_NSLOTS
};

// kernels timed by the profiling hook (kde_profile_enable / kde_profile_read)
enum KdeProfId { PROF_CV_PAIRS = 0, PROF_DEPOSIT, PROF_GATHER, PROF_SORT, PROF_POISSON, PROF_CV_GRID, PROF_CV_LOO,
                 PROF_SPECTRAL, PROF_AD, PROF_DEPOSIT_ROWS, PROF_NIDS };

struct kde_ctx {
    int device = 0;
    // profiling: event pairs recorded around selected launches while enabled
    bool prof_on = false;
    long long launches = 0;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof;
    std::vector<cudaEvent_t> ev_pool;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    std::string err;
    unsigned int *d_status = nullptr;  // [0] code, [1] detail, [2], [3] spare
    void *ws[WS_NSLOTS] = {};
    size_t ws_bytes[WS_NSLOTS] = {};
    // cached tables keyed by (Ng, precision): half-angle sines/cosines of the nodes
    std::map<std::pair<int, int>, void *> node_tab;
    // cached Green's functions keyed by (Ng, L bits, fd, precision)
    std::map<std::tuple<int, uint64_t, int, int>, void *> green_tab;
    // Anderson-Darling per-bin logarithms (one table per context)
    void *ad_tab = nullptr;
    float2 *norm_tab = nullptr;  // FP32 width-normalisation table (kde_norm_tab), built at creation
    unsigned wait_polls = 1u << 26;         // polls of a bounded device wait (kde_set_wait_limit)
    bool count_flip = false;                // which sort count table the next counted sort reads (sort.cu)
    bool autotune = false;                  // kde_set_autotune
    bool overlap = true;                    // kde_set_launch_overlap: PDL launches in the step chain
    std::map<uint64_t, int> gat2_tuned;     // packed-gather tile shape per key (gather.cu)
    double cut_fixed = 0.0;                 // kde_set_truncation: FP32 cut exponent, 0 = automatic
    std::map<uint64_t, float> cut_tuned;    // FP32 PIC truncation cut exponent per key (pic.cu)
    void *sp_atab = nullptr;                // workspace holding the Bessel ratios of sp_atab_cands (spectral.cu)
    std::vector<double> sp_atab_cands;
};

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
kde_status kde_fail(kde_ctx *ctx, kde_status code, const char *fmt, ...);
kde_status kde_cuda_check(kde_ctx *ctx, cudaError_t e, const char *what);
void *kde_ws(kde_ctx *ctx, WsSlot slot, size_t bytes);  // grows the slot; nullptr + error on failure
const void *kde_node_table(kde_ctx *ctx, int Ng, bool f64);
const void *kde_green_table(kde_ctx *ctx, int Ng, double L, bool fd, bool f64);
double kde_host_i0e(double x);  // scaled Bessel I0e in FP64 on the host (uniform widths)

#define KDE_TRY(expr)                       \
    do {                                    \
        kde_status _s = (expr);             \
        if (_s != KDE_OK) return _s;        \
    } while (0)
#define KDE_CUDA(ctx, expr, what)                                   \
    do {                                                            \
        cudaError_t _e = (expr);                                    \
        if (_e != cudaSuccess) return kde_cuda_check(ctx, _e, what); \
    } while (0)
#define KDE_LAUNCHED(ctx, what)                        \
    do {                                               \
        ++(ctx)->launches;                             \
        KDE_CUDA(ctx, cudaGetLastError(), what);       \
    } while (0)

// launch on the context's stream; with `pdl` and the context's overlap setting on, the
// kernel may begin while the previous kernel in the stream runs (see kde_pdl_wait)
template <typename... KArgs, typename... Args>
inline cudaError_t kde_launch(kde_ctx *ctx, bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = (pdl && ctx->overlap) ? 1u : 0u;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// profiling hook: when enabled, records an event pair around a launch on the
// context's stream
cudaEvent_t kde_prof_event(kde_ctx *ctx);
struct KdeProfScope {
    kde_ctx *c;
    int id;
    cudaEvent_t b = nullptr;
    KdeProfScope(kde_ctx *ctx, int i) : c(ctx), id(i)
    {
        if (c->prof_on) {
            b = kde_prof_event(c);
            cudaEventRecord(b, c->stream);
        }
    }
    ~KdeProfScope()
    {
        if (b) {
            cudaEvent_t e = kde_prof_event(c);
            cudaEventRecord(e, c->stream);
            c->prof.push_back({id, {b, e}});
        }
    }
};

// NVTX range around the host-side launches of one stage (sort, deposit, Poisson,
// gather + push, width update, CV pieces), so that a profiler's timeline groups
// each stage's kernels; without a profiler attached the calls do nothing
struct KdeRange {
    explicit KdeRange(const char *name) { nvtxRangePushA(name); }
    ~KdeRange() { nvtxRangePop(); }
    KdeRange(const KdeRange &) = delete;
    KdeRange &operator=(const KdeRange &) = delete;
};

// FP32 truncation: each kernel is evaluated over at least the nodes where its weight is
// 2^-xcut of its peak or more.  xcut = 24 unless fixed by kde_set_truncation (or, for
// the PIC step, chosen by the truncation tuner); FP64 paths always use KDE_XCUT64.
inline float kde_fp32_cut(const kde_ctx *ctx)
{
    return ctx->cut_fixed > 0.0 ? (float)ctx->cut_fixed : (float)KDE_XCUT;
}

// autotuner key: grid size, log2 of N, and the uniform width in quarter octaves (0 for
// per-particle widths, whose values the host does not see)
inline uint64_t kde_width_key(int64_t N, int Ng, bool per_particle, double kappa_u)
{
    int lg = 0;
    while (lg < 40 && (1LL << (lg + 1)) <= N) ++lg;
    int kc = 0;
    if (!per_particle) {
        const double q = 4.0 * log2(kappa_u) + 128.0;
        kc = q < 1.0 ? 1 : (q > 255.0 ? 255 : (int)q);
    }
    return (uint64_t)Ng | ((uint64_t)lg << 16) | ((uint64_t)kc << 24);
}

// number of nodes on each side of a particle's cell that its truncated kernel
// can reach: ceil(r / dtheta), r = 2 asin(sqrt(XCUT ln2 / (2 kappa))), or Ng
// when the support is the whole circle
__host__ __device__ inline int kde_window_nodes(double kappa, int Ng)
{
    double s2 = KDE_XCUT * KDE_LN2 / (2.0 * kappa);
    if (s2 >= 1.0) return Ng;
    double r = 2.0 * asin(sqrt(s2));
    double w = ceil(r * Ng / KDE_TWO_PI);
    return w >= Ng ? Ng : (int)w;
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float kde_ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double kde_ex2(double x) { return exp2(x); }

// packed FP32 pairs (f32x2: one instruction applies the operation to both lanes)
typedef unsigned long long kde_f2;
__device__ __forceinline__ kde_f2 kde_pk(float a, float b)
{
    kde_f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void kde_upk(kde_f2 r, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ kde_f2 kde_mul2(kde_f2 a, kde_f2 b)
{
    kde_f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ kde_f2 kde_fma2(kde_f2 a, kde_f2 b, kde_f2 c)
{
    kde_f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// 2^(-x) for both lanes of a packed pair
__device__ __forceinline__ kde_f2 kde_ex2neg2(kde_f2 x)
{
    float a, b;
    kde_upk(x, a, b);
    return kde_pk(kde_ex2(-a), kde_ex2(-b));
}
// 2^x for both lanes of a packed pair
__device__ __forceinline__ kde_f2 kde_ex22(kde_f2 x)
{
    float a, b;
    kde_upk(x, a, b);
    return kde_pk(kde_ex2(a), kde_ex2(b));
}

// largest width for the cosine form of the FP32 kernel value,
// 2^(K cos x_j cos x_g + K sin x_j sin x_g - K) with K = kappa log2(e): three
// multiply-adds per pair instead of the half-angle form's four, at the price of an
// exponent that carries about K 2^-24 of cancellation error near the peak (a
// relative error of about 2e-8 kappa in the L2 norm of a density)
#define KDE_COSFORM_KMAX 32.0f

__device__ __forceinline__ void kde_flag(unsigned int *status, unsigned code, unsigned detail)
{
    if (status && atomicCAS(status, 0u, code) == 0u) status[1] = detail;
}

// Programmatic dependent launch.  A kernel launched by kde_launch with overlap on may
// start while the kernel before it in the stream is still running.  Every kernel so
// launched keeps two rules:
//  * every CTA executes kde_pdl_wait() before it reads anything the previous kernel
//    writes, before its first global write (the device status word, which only ever
//    goes from zero to an error code, excepted) and before it exits; the wait returns
//    once the previous grid has completed and its writes are visible (at once without
//    PDL);
//  * kde_pdl_trigger(), which lets the next kernel start, comes after kde_pdl_wait().
// So when a kernel starts, the kernel two places before it has completed, and data
// written two or more kernels back may be read before the wait.
__device__ __forceinline__ void kde_pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void kde_pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// half-angle sine and cosine of the position code: theta / 2 = pi u / 2^32.
// FP32: the code is split as u = hi 2^16 + lo; sincospif of the exact float
// hi 2^-16 gives the angle of hi, and the angle-sum identity adds that of lo.
__device__ __forceinline__ void kde_half_sincos(uint32_t u, float &s, float &c)
{
    // the low part is an angle d = pi lo 2^-32 < 4.8e-5: sin d = d (1 - d^2 / 6) and
    // cos d = 1 - d^2 / 2 round to d and 1 in FP32 (d^2 / 2 < 1.2e-9 is below half an
    // ulp of 1), so the angle sum needs no second sine/cosine evaluation
    float sh, ch;
    sincospif((float)(u >> 16) * (1.0f / 65536.0f), &sh, &ch);
    const float d = (float)(u & 0xFFFFu) * (float)(KDE_PI / 4294967296.0);
    s = fmaf(ch, d, sh);
    c = fmaf(-sh, d, ch);
}
__device__ __forceinline__ void kde_half_sincos(uint32_t u, double &s, double &c)
{
    sincospi((double)u * (1.0 / 4294967296.0), &s, &c);
}

// cell index of a position on an Ng-node grid: floor(u Ng / 2^32)
__device__ __forceinline__ int kde_cell(uint32_t u, int Ng)
{
    return (int)(((uint64_t)u * (uint64_t)Ng) >> 32);
}

// scaled modified Bessel function I0e(x) = exp(-x) I0(x) in FP64 (power series
// below 30, Hankel asymptotic expansion above)
__host__ __device__ inline double kde_i0e(double x)
{
    if (x < 0) x = -x;
    if (x < 30.0) {
        double q = 0.25 * x * x, term = 1.0, sum = 1.0;
        for (int k = 1; k < 200; ++k) {
            term *= q / ((double)k * (double)k);
            sum += term;
            if (term < 1e-17 * sum) break;
        }
        return sum * exp(-x);
    }
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 60; ++k) {
        double nx = term * (2.0 * k - 1.0) * (2.0 * k - 1.0) / (8.0 * x * k);
        if (nx >= term) break;
        term = nx;
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum / sqrt(KDE_TWO_PI * x);
}

// von Mises normalisation 1 / (2 pi I0e(kappa))
__host__ __device__ inline double kde_norm(double kappa) { return 1.0 / (KDE_TWO_PI * kde_i0e(kappa)); }

// FP32 von Mises normalisation from a table built once per context:
// norm(kappa) = 1 / (2 pi I0e(kappa)) = sqrt(1 + 2 pi kappa) / (2 pi q(kappa)) with
// q(kappa) = I0e(kappa) sqrt(1 + 2 pi kappa), which is smooth in t = ln kappa and
// runs from 1 (kappa -> 0) through a maximum of 1.31 back to 1 (kappa -> infinity).
// The table holds q and h dq/dt (FP64-computed, stored FP32) at t = KDE_NTAB_T0 + i h,
// h = 1/32, from kappa = 9.7e-10 to 1.02e6; cubic Hermite interpolation.  Relative
// error below 5e-7 over (0, 1e6] (FP32 evaluation; the FP64 norm rounded to FP32
// is within 6e-8), which keeps FP64 Bessel series off the per-particle paths.
#define KDE_NTAB_N 1108
#define KDE_NTAB_T0 (-20.75)
#define KDE_NTAB_INVH 32.0
__device__ __forceinline__ float kde_norm_tab(const float2 *__restrict__ tab, float kappa)
{
    const float u = (logf(kappa) - (float)KDE_NTAB_T0) * (float)KDE_NTAB_INVH;
    float q = 1.f;  // below the table, q = 1 + (pi - 1) kappa to within 2e-9
    if (u > 0.f) {
        const int i = min((int)u, KDE_NTAB_N - 2);
        const float s = u - (float)i, r = 1.f - s;
        const float2 a = tab[i], b = tab[i + 1];
        // Hermite basis on [0, 1]
        const float h00 = (1.f + 2.f * s) * r * r, h10 = s * r * r, h01 = s * s * (3.f - 2.f * s), h11 = -s * s * r;
        q = fmaf(h00, a.x, fmaf(h10, a.y, fmaf(h01, b.x, h11 * b.y)));
    }
    return sqrtf(fmaf((float)KDE_TWO_PI, kappa, 1.f)) / ((float)KDE_TWO_PI * q);
}

// exact power-of-two scale for the int64 fixed-point grid accumulators: the
// largest possible node value is `bound`, kept below 2^62
__host__ __device__ inline double kde_acc_scale(double bound)
{
    int e;
    frexp(bound > 0 ? bound : 1.0, &e);  // bound < 2^e
    return ldexp(1.0, 62 - e);
}

// ---------------------------------------------------------------------------
// internal launchers (defined in the kernel translation units)
// ---------------------------------------------------------------------------
// counting sort by bin = floor(u nbins / 2^32), stable.  Moves u and up to four
// payload arrays (element size 4 or 8 bytes); writes the source index of every
// output slot to perm_out when not null.
struct SortPayload {
    const void *src;
    void *dst;
    int elem;
};
kde_status kde_sort_by_bin(kde_ctx *ctx, const uint32_t *u, int64_t N, int nbins, uint32_t *u_out,
                           const SortPayload *pl, int npl, uint32_t *perm_out, bool counted = false);
// the count table of such a sort (bin-major: entry bin * nblk + tile, tile = index >>
// tile_shift), for a kernel that adds the counts of the keys it writes; with
// counted = true kde_sort_by_bin uses the table as it stands (every sort leaves it zero)
struct SortCounts {
    unsigned int *counts;
    int nblk;
    int tile_shift;
};
kde_status kde_sort_counts_table(kde_ctx *ctx, int64_t N, int nbins, SortCounts *out);
// standard-PIC shapes inside pic_step: deposit of the B-spline shape (degree
// order, width h) into int64 accumulators acc[Ng] (zeroed here; *bound_out = the
// largest possible node value), and gather + leap-frog push in place
kde_status kde_bspline_deposit_acc(kde_ctx *ctx, const uint32_t *u, int64_t N, int order, double h, int Ng, double L,
                                   long long *acc, double *bound_out);
kde_status kde_bspline_gather_push(kde_ctx *ctx, uint32_t *u, float *v, int64_t N, int order, double h, int Ng,
                                   double L, const float *E, double kick_qm_dt, double dt_scale);
// ascending sort of N 32-bit codes (LSD radix, four stable 8-bit passes);
// tmp: N-element scratch; u may alias neither out nor tmp
kde_status kde_radix_sort_u32(kde_ctx *ctx, const uint32_t *u, int64_t N, uint32_t *out, uint32_t *tmp);

// deposit of cell-sorted particles into int64 accumulators acc[Ng] (zeroed
// here).  Particle j contributes w_j * coef * norm_j * exp(-2 kappa_j sin^2(..)).
// Arrays may be null (then the uniform scalar is used; norm null with a kappa
// array means "compute the norm from the width").  `bound` is the largest
// possible node value; with wmax_bits it is N * coef * norm_bound * w_max.
template <typename T>
kde_status kde_deposit_sorted(kde_ctx *ctx, const uint32_t *u, const T *kappa, T kappa_u, const T *norm, T norm_u,
                              const T *w, T w_u, int64_t N, int Ng, double coef, long long *acc, double bound,
                              const unsigned int *wmax_bits, double norm_bound);
template <typename T>
kde_status kde_acc_to_real(kde_ctx *ctx, const long long *acc, int Ng, double bound, const unsigned int *wmax_bits,
                           double wscale, T *out);
// grows the workspace of the FP32 deposit for N particles on Ng nodes (kde_reserve)
kde_status kde_deposit_reserve(kde_ctx *ctx, int64_t N, int Ng);
// the FP32 deposit of cell-sorted particles (uniform weight w_u, N >= 1) left as its
// per-CTA int64 rows (workspace, valid until the next deposit on the context):
// node g of row k is rows[k Ng + ((g - hdr[k].x) mod Ng)] when that index is below
// hdr[k].y, else 0; fixed-point scale kde_acc_scale(bound)
struct DepRows {
    const long long *rows;
    const int2 *hdr;
    int G;
};
kde_status kde_deposit_rows_f32(kde_ctx *ctx, const uint32_t *u, const float *kappa, float kappa_u, const float *norm,
                                float norm_u, int64_t N, int Ng, double coef, float w_u, double bound, DepRows *out,
                                float xcut = 0.f);
// the PIC step's field from those rows: rho_total = background + charge * rho with its
// mean removed (so the constant background drops out), E by the spectral or
// finite-difference Green's function (FP32 output)
kde_status kde_field_from_rows(kde_ctx *ctx, const long long *rows, const int2 *hdr, int G, int Ng, double L,
                               double acc_inv, double charge, bool fd, float *E_out);

// Poisson solve of rho_total = background + charge * rho, rho given as a real
// array or as int64 accumulators (value = acc * acc_inv)
template <typename T>
kde_status kde_poisson_impl(kde_ctx *ctx, const T *rho, const long long *acc, double acc_inv, int Ng, double L,
                            double charge, double background, bool fd, T *E_out);
template <typename T>
kde_status kde_energy_impl(kde_ctx *ctx, const T *E, int Ng, double L, double *energy_out);

struct PushArgs {
    const void *v_in;        // sorted velocities
    uint32_t *u_out;         // updated positions (sorted order)
    void *v_out;
    void *kappa_out;         // widths written back (sorted order), or null
    const void *norm_in;
    void *norm_out;
    const uint32_t *id_in;
    uint32_t *id_out;
    double kick;             // velocity kick factor (1/2 on the first step)
    double qm_dt;
    double dt_scale;         // dt * 2^32 / L
    double *energy;          // field energy slot for this step, or null
    const double *kstar_in;  // CV width in force (device), or null for the uniform width
    double *kstar_out;
    double dx;
    unsigned int *counts;    // FP32 gather: count table of the next cell sort (kde_sort_counts_table), or null
    int cnt_nblk, cnt_shift;
    float xcut;              // FP32 truncation cut exponent (kde_fp32_cut), 0: the context's default
};
template <typename T>
kde_status kde_gather_sorted(kde_ctx *ctx, const uint32_t *u, const T *kappa, T kappa_u, const T *norm, T norm_u,
                             int64_t N, const T *field, int Ng, double coef, T *out, const uint32_t *perm,
                             const PushArgs *push, float xcut = 0.f);

// candidate widths (or scale factors) for the CV kernels, passed by value
struct CandList {
    int n;
    int scale_mode;
    double k[256];
};

// CV on the device without host synchronisation.  u: positions (any order);
// cand_host: host float64[n_cand] in the caller's order.  Results stay on the
// device: cv_dev float64[n_cand] (caller's order), argmin_dev int32, loo
// (float32, order of u, at the argmin) when not null, kstar_dev float64 (the
// selected candidate) when not null.
kde_status kde_cv_device(kde_ctx *ctx, const uint32_t *u, const float *kappa_rel, int64_t N, double L,
                         const double *cand_host, int n_cand, bool scale_mode, double *cv_dev, int *argmin_dev,
                         float *loo, double *kstar_dev);

// Anderson-Darling test (Sec. II.D) of positions u (any order) against the
// uniform distribution: out_dev[0] = A^2, out_dev[1] = ln p; ln p also to
// *lp_slot when not null.  Stream-ordered.
kde_status kde_ad_device(kde_ctx *ctx, const uint32_t *u, int64_t N, double *out_dev, double *lp_slot);

// leave-one-out densities at the width cand[*argmin_dev] (caller's order) by the
// exact Fourier form: the same values as the pair-sum pass, O(N M(kappa*)) work
kde_status kde_loo_spectral_device(kde_ctx *ctx, const uint32_t *u, int64_t N, double L, const double *cand_host,
                                   int n_cand, const int *argmin_dev, float *loo);
int kde_spec_modes(double kappa);  // Fourier modes the exact form keeps for a width
// the cost rule between the exact forms of a uniform-width CV curve (true: Fourier form)
bool kde_cv_prefer_spectral(int64_t N, const double *cand, int n_cand);

// the same results by the exact Fourier form (uniform widths only)
kde_status kde_cv_spectral_device(kde_ctx *ctx, const uint32_t *u, int64_t N, double L, const double *cand_host,
                                  int n_cand, double *cv_dev, int *argmin_dev, float *loo, double *kstar_dev);

// Silverman widths from leave-one-out densities; kstar from the device when
// kstar_dev is not null.  Writes widths (and norms when norm_out is not null)
// as float or double.
kde_status kde_adapt_device(kde_ctx *ctx, const float *loo, int64_t N, double L, const double *kstar_dev,
                            double kstar_host, double alpha, double kmin, double kmax, void *kappa_out,
                            void *norm_out, bool f64);
