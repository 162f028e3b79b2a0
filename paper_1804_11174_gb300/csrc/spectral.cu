// spectral.cu -- exact Fourier-space evaluation of the leave-one-out CV
// (Sec. II.B, Eq. cv_def) for a uniform width.
//
// The von Mises kernel is K(t) = (1/2pi) sum_m A_m e^{imt}, A_m = I_m/I_0.
// With the structure factor S_m = sum_j e^{i m theta_j}:
//   sum_{i,j} K(theta_i - theta_j) = (1/2pi) (n^2 + 2 sum_{m>=1} A_m |S_m|^2)
//   int fhat^2                     = (1/(2pi n^2)) (n^2 + 2 sum_{m>=1} A_m^2 |S_m|^2)
//   n K(0)                         = n norm(kappa)
//   sum_j K(theta_i - theta_j)     = (1/2pi) (n + 2 sum_{m>=1} A_m Re(e^{i m theta_i} conj(S_m)))
// These are identities; modes are cut where A_m < 1e-17.  The cost is
// O(N M) for S_m (M ~ sqrt(78 kappa_max)) instead of O(N^2) pairs per
// candidate, and all candidates share one S_m.
//
// Phases are exact: m theta_j = 2 pi (m u_j mod 2^32) / 2^32 in integer
// arithmetic, then one FP32 sincospi for the first of every four consecutive
// modes and a rotation by e^{i theta_j} for the next three (an ulp or two each).
// Sub-chunk sums run in FP32 and are
// combined in FP64 in a fixed order; the CV combination and the leave-one-out
// sums are FP64.  Particles may come in any order (no sort).
#include "common.cuh"

#define SP_THREADS 256
#define SP_SUB 256
#define SP_MAXM 16384
#define SP_MAXCHUNK 16384
#define SP_Q 8         // consecutive modes a thread in the structure factor
#define SP_SF_THREADS 128  // threads of a structure-factor block (SP_Q SP_SF_THREADS modes)

// modes needed for a width: A_m ~ exp(-m^2 / (2 kappa)) < 1e-17 beyond sqrt(78.4 kappa)
__host__ __device__ inline int spec_modes(double kappa)
{
    int M = (int)ceil(sqrt(78.4 * kappa)) + 8;
    return M > SP_MAXM ? SP_MAXM : M;
}

// A_m(kappa), m = 0..M, into A[0..M]; r scratch of M + tail + 1 doubles.
// Backward recurrence r_m = 1 / (2m/kappa + r_{m+1}) for r_m = I_m / I_{m-1},
// started at index M + 64 + 2 sqrt(kappa) from the estimate
// kappa / (m + 1/2 + sqrt((m + 1/2)^2 + kappa^2)), then A_m = r_1 ... r_m.
__device__ void spec_ratios(double kappa, int M, double *A)
{
    const int start = M + 64 + (int)(2.0 * sqrt(kappa));
    double r = kappa / (start + 0.5 + sqrt((start + 0.5) * (start + 0.5) + kappa * kappa));
    for (int m = start; m > M; --m) r = 1.0 / (2.0 * m / kappa + r);
    // now r = r_{M+1}; store r_m for m = M..1 in A[m]
    for (int m = M; m >= 1; --m) {
        r = 1.0 / (2.0 * m / kappa + r);
        A[m] = r;
    }
    A[0] = 1.0;
    for (int m = 1; m <= M; ++m) A[m] *= A[m - 1];
}

// structure factor partials: block (chunk, mode block); thread = SP_Q consecutive
// modes m0 .. m0 + SP_Q - 1: one exact-phase sincospi for m0, then each further mode by
// a rotation with e^{i theta_j} (tabulated per particle in shared memory), which costs
// four FP32 operations instead of a sincospi and adds at most an ulp or two per step.
// The partials are laid out with stride M; modes above *mlim (when given) are skipped.
__global__ void __launch_bounds__(SP_SF_THREADS)
    spec_sf_kernel(const uint32_t *__restrict__ u, int64_t N, int64_t chunk, int M, const int *mlim, double2 *part)
{
    extern __shared__ __align__(8) uint32_t us[];
    float2 *e1 = (float2 *)(us + ((chunk + 1) & ~1LL));  // (cos, sin) of theta_j
    const int Me = mlim ? min(M, *mlim) : M;
    const int mb = 1 + (int)blockIdx.y * SP_SF_THREADS * SP_Q;
    if (mb > Me) return;  // the whole mode block is above the limit
    const int64_t j0 = (int64_t)blockIdx.x * chunk;
    const int n = (int)(N - j0 < chunk ? N - j0 : chunk);
    for (int k = threadIdx.x; k < n; k += SP_SF_THREADS) {
        const uint32_t uk = u[j0 + k];
        us[k] = uk;
        float s1, c1;
        sincospif((float)(int32_t)uk * (1.0f / 2147483648.0f), &s1, &c1);
        e1[k] = make_float2(c1, s1);
    }
    __syncthreads();
    const int m0 = mb + threadIdx.x * SP_Q;
    if (m0 > Me) return;
    double cr[SP_Q], ci[SP_Q];
#pragma unroll
    for (int q = 0; q < SP_Q; ++q) cr[q] = ci[q] = 0.0;
    for (int k0 = 0; k0 < n; k0 += SP_SUB) {
        const int k1 = k0 + SP_SUB < n ? k0 + SP_SUB : n;
        float fr[SP_Q], fi[SP_Q];
#pragma unroll
        for (int q = 0; q < SP_Q; ++q) fr[q] = fi[q] = 0.f;
#pragma unroll 2
        for (int k = k0; k < k1; ++k) {
            const uint32_t ph = (uint32_t)m0 * us[k];  // m0 theta / (2 pi) in 2^-32 turns
            float s, c;
            sincospif((float)(int32_t)ph * (1.0f / 2147483648.0f), &s, &c);
            const float2 e = e1[k];
            fr[0] += c;
            fi[0] += s;
#pragma unroll
            for (int q = 1; q < SP_Q; ++q) {
                const float cn = fmaf(c, e.x, -s * e.y), sn = fmaf(s, e.x, c * e.y);
                c = cn;
                s = sn;
                fr[q] += c;
                fi[q] += s;
            }
        }
#pragma unroll
        for (int q = 0; q < SP_Q; ++q) {
            cr[q] += (double)fr[q];
            ci[q] += (double)fi[q];
        }
    }
#pragma unroll
    for (int q = 0; q < SP_Q; ++q)
        if (m0 + q <= Me) part[(size_t)blockIdx.x * M + (m0 + q - 1)] = make_double2(cr[q], ci[q]);
}

// S_m = sum over the chunks (modes up to *mlim when given) in a fixed order, in two
// stages: block (32 modes, chunk group g) -- warp w adds chunks c0 + w, c0 + w + 8, ...
// of the group in order, then the eight warp sums in warp order -- and then the
// SPR_G group sums in group order
#define SPR_G 8
__global__ void __launch_bounds__(256) spec_reduce_kernel(const double2 *part, int nchunks, int M, const int *mlim,
                                                          double2 *gpart)
{
    __shared__ double2 ws[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Me = mlim ? min(M, *mlim) : M;
    const int m = (int)blockIdx.x * 32 + lane;
    const int c0 = (int)((int64_t)nchunks * blockIdx.y / SPR_G), c1 = (int)((int64_t)nchunks * (blockIdx.y + 1) / SPR_G);
    double sr = 0.0, si = 0.0;
    if (m < Me) {
#pragma unroll 4
        for (int c = c0 + warp; c < c1; c += 8) {
            const double2 p = part[(size_t)c * M + m];
            sr += p.x;
            si += p.y;
        }
    }
    ws[warp][lane] = make_double2(sr, si);
    __syncthreads();
    if (warp == 0 && m < Me) {
        double2 t = ws[0][lane];
#pragma unroll
        for (int w = 1; w < 8; ++w) {
            t.x += ws[w][lane].x;
            t.y += ws[w][lane].y;
        }
        gpart[(size_t)blockIdx.y * M + m] = t;
    }
}

__global__ void spec_reduce2_kernel(const double2 *gpart, int M, const int *mlim, double2 *S)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= (mlim ? min(M, *mlim) : M)) return;
    double2 t = gpart[m];
#pragma unroll
    for (int g = 1; g < SPR_G; ++g) {
        const double2 p = gpart[(size_t)g * M + m];
        t.x += p.x;
        t.y += p.y;
    }
    S[m] = t;
}

// one CTA per candidate (caller's order): Bessel ratios (sequential recurrence,
// one thread; skipped when Atab already holds this candidate list's ratios), then the
// three mode sums over the block and CV (x units)
__global__ void __launch_bounds__(SP_THREADS)
    spec_cv_kernel(const double2 *S, CandList cl, int64_t N, double L, int Astride, double *Atab, int ratios_ready,
                   double *cv_out)
{
    __shared__ double r0[SP_THREADS], r1[SP_THREADS], r2[SP_THREADS];
    const int c = blockIdx.x;
    const double n = (double)N;
    const double kappa = cl.k[c];
    const int M = spec_modes(kappa);
    double *A = Atab + (size_t)c * Astride;
    if (threadIdx.x == 0 && !ratios_ready) spec_ratios(kappa, M, A);
    __syncthreads();
    double sA = 0.0, sAS = 0.0, sA2S = 0.0;
    for (int m = 1 + threadIdx.x; m <= M; m += SP_THREADS) {
        const double2 s = S[m - 1];
        const double p = s.x * s.x + s.y * s.y;
        const double a = A[m];
        sA += a;
        sAS += a * p;
        sA2S += a * a * p;
    }
    r0[threadIdx.x] = sA;
    r1[threadIdx.x] = sAS;
    r2[threadIdx.x] = sA2S;
    __syncthreads();
    for (int o = SP_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            r0[threadIdx.x] += r0[threadIdx.x + o];
            r1[threadIdx.x] += r1[threadIdx.x + o];
            r2[threadIdx.x] += r2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double f2 = (n * n + 2.0 * r2[0]) / (KDE_TWO_PI * n * n);
        const double pairs = (n * n + 2.0 * r1[0] - n - 2.0 * n * r0[0]) / KDE_TWO_PI;
        cv_out[c] = (KDE_TWO_PI / L) * (f2 - 2.0 * pairs / (n * (n - 1.0)));
    }
}

// argmin (smallest index on ties) and the selected width
__global__ void spec_argmin_kernel(const double *cv, CandList cl, int *argmin, double *kstar)
{
    int best = 0;
    for (int q = 1; q < cl.n; ++q)
        if (cv[q] < cv[best]) best = q;
    *argmin = best;
    if (kstar) *kstar = cl.k[best];
}

// the selected width kappa* = cand[*argmin]: its mode count, Bessel ratios A[0..M]
// and normalisation 1 / (2 pi I0e(kappa*)), for the leave-one-out pass
struct SpecSel {
    int M;
    double norm;
    const double *A;  // the ratios A[0..M]: a row of the candidates' table, or the kernel's own output
};
// Atab: the candidates' ratio table (row stride Astride) when the caller has it, else
// nullptr and the ratios are worked out into A
__global__ void spec_select_kernel(CandList cl, const int *argmin, SpecSel *sel, double *A, const double *Atab,
                                   int Astride)
{
    const double kappa = cl.k[*argmin];
    const int M = spec_modes(kappa);
    if (Atab) {
        sel->A = Atab + (size_t)*argmin * Astride;
    } else {
        spec_ratios(kappa, M, A);
        sel->A = A;
    }
    sel->M = M;
    sel->norm = kde_norm(kappa);
}

// A_m S_m in FP32 for the leave-one-out sums
__global__ void spec_as_kernel(const double2 *S, const SpecSel *sel, float2 *AS)
{
    const int m = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    if (m > sel->M) return;
    const double *A = sel->A;
    const double2 s = S[m - 1];
    AS[m - 1] = make_float2((float)(A[m] * s.x), (float)(A[m] * s.y));
}

// leave-one-out density at the selected width for every particle (input order):
// sum_j K(theta_i - theta_j) = (1/2pi)(n + 2 sum_m Re(e^{i m theta_i} conj(A_m S_m))),
// minus the particle's own K(0).  Exact integer phases, FP32 terms with compensated
// (Kahan) summation over the modes; the combination in FP64 once per particle.
#define SP_LOO_CH 1024
__global__ void __launch_bounds__(SP_THREADS)
    spec_loo_kernel(const uint32_t *__restrict__ u, int64_t N, const float2 *__restrict__ AS,
                    const SpecSel *__restrict__ sel, double xs, float *loo)
{
    __shared__ float2 sAS[SP_LOO_CH];
    const int M = sel->M;
    const int64_t i = (int64_t)blockIdx.x * SP_THREADS + threadIdx.x;
    const uint32_t ui = i < N ? u[i] : 0u;
    float acc = 0.f, comp = 0.f;
    for (int m0 = 1; m0 <= M; m0 += SP_LOO_CH) {
        const int cnt = M - m0 + 1 < SP_LOO_CH ? M - m0 + 1 : SP_LOO_CH;
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += SP_THREADS) sAS[k] = AS[m0 - 1 + k];
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < cnt; ++k) {
            const uint32_t ph = (uint32_t)(m0 + k) * ui;
            float s, co;
            sincospif((float)(int32_t)ph * (1.0f / 2147483648.0f), &s, &co);
            const float2 q = sAS[k];
            // Re(e^{i m theta_i} conj(A_m S_m)) = cos * Re + sin * Im, added with compensation
            const float y = fmaf(co, q.x, s * q.y) - comp;
            const float t = acc + y;
            comp = (t - acc) - y;
            acc = t;
        }
    }
    if (i >= N) return;
    const double n = (double)N;
    const double all = (n + 2.0 * ((double)acc - (double)comp)) / KDE_TWO_PI;
    loo[i] = (float)(xs * (all - sel->norm) / (n - 1.0));
}

// leave-one-out densities at cand[*argmin] from the structure factor S (modes
// 1..M(kappa*) present)
static kde_status spec_loo_from_S(kde_ctx *ctx, const uint32_t *u, int64_t N, double L, const double2 *S,
                                  const CandList &cl, int Mmax, const int *argmin_dev, float *loo,
                                  const double *Atab = nullptr, int Astride = 0)
{
    double *Asel = (double *)kde_ws(ctx, WS_SP_ASEL, (size_t)(Mmax + 1) * 8 + 64);
    float2 *AS = (float2 *)kde_ws(ctx, WS_SP_AS, (size_t)Mmax * sizeof(float2) + 64);
    SpecSel *sel = (SpecSel *)kde_ws(ctx, WS_SP_SEL, sizeof(SpecSel));
    if (!Asel || !AS || !sel) return KDE_ENOMEM;
    spec_select_kernel<<<1, 1, 0, ctx->stream>>>(cl, argmin_dev, sel, Asel, Atab, Astride);
    KDE_LAUNCHED(ctx, "spec_select_kernel");
    spec_as_kernel<<<(Mmax + 255) / 256, 256, 0, ctx->stream>>>(S, sel, AS);
    KDE_LAUNCHED(ctx, "spec_as_kernel");
    {
        KdeProfScope _ps(ctx, PROF_CV_LOO);
        spec_loo_kernel<<<(unsigned)((N + SP_THREADS - 1) / SP_THREADS), SP_THREADS, 0, ctx->stream>>>(
            u, N, AS, sel, KDE_TWO_PI / L, loo);
    }
    KDE_LAUNCHED(ctx, "spec_loo_kernel");
    return KDE_OK;
}

// structure factor for modes 1..M (or up to *mlim) into S
static kde_status spec_structure(kde_ctx *ctx, const uint32_t *u, int64_t N, int M, const int *mlim, double2 **S_out)
{
    // about a thousand chunks keep every SM busy; the partials stay under 2^22 entries (64 MB)
    int64_t chunk = 1024;
    while (((N + chunk - 1) / chunk > 1024 || (N + chunk - 1) / chunk * M > (1 << 22)) && chunk < SP_MAXCHUNK)
        chunk *= 2;
    const int nchunks = (int)((N + chunk - 1) / chunk);
    double2 *part = (double2 *)kde_ws(ctx, WS_SP_PART, (size_t)(nchunks + SPR_G) * M * sizeof(double2));
    double2 *gpart = part + (size_t)nchunks * M;  // the chunk groups' sums
    double2 *S = (double2 *)kde_ws(ctx, WS_SP_S, (size_t)M * sizeof(double2));
    if (!part || !S) return KDE_ENOMEM;
    static bool attr = false;
    if (!attr) {
        KDE_CUDA(ctx, cudaFuncSetAttribute(spec_sf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           SP_MAXCHUNK * 12 + 8),
                 "spec_sf_kernel attribute");
        attr = true;
    }
    {
        KdeProfScope _ps(ctx, PROF_SPECTRAL);
        dim3 grid((unsigned)nchunks, (unsigned)((M + SP_SF_THREADS * SP_Q - 1) / (SP_SF_THREADS * SP_Q)));
        spec_sf_kernel<<<grid, SP_SF_THREADS, (size_t)((chunk + 1) & ~1LL) * 4 + (size_t)chunk * 8, ctx->stream>>>(
            u, N, chunk, M, mlim, part);
    }
    KDE_LAUNCHED(ctx, "spec_sf_kernel");
    spec_reduce_kernel<<<dim3((unsigned)((M + 31) / 32), SPR_G), 256, 0, ctx->stream>>>(part, nchunks, M, mlim, gpart);
    KDE_LAUNCHED(ctx, "spec_reduce_kernel");
    spec_reduce2_kernel<<<(M + 255) / 256, 256, 0, ctx->stream>>>(gpart, M, mlim, S);
    KDE_LAUNCHED(ctx, "spec_reduce2_kernel");
    *S_out = S;
    return KDE_OK;
}

// selected width's mode count, for the structure factor of the leave-one-out pass
__global__ void spec_mlim_kernel(CandList cl, const int *argmin, int *mlim) { *mlim = spec_modes(cl.k[*argmin]); }

kde_status kde_loo_spectral_device(kde_ctx *ctx, const uint32_t *u, int64_t N, double L, const double *cand_host,
                                   int n_cand, const int *argmin_dev, float *loo)
{
    CandList cl{};
    cl.n = n_cand;
    double kmax = 0.0;
    for (int c = 0; c < n_cand; ++c) {
        cl.k[c] = cand_host[c];
        kmax = cand_host[c] > kmax ? cand_host[c] : kmax;
    }
    const int Mmax = spec_modes(kmax);
    int *mlim = (int *)kde_ws(ctx, WS_SP_MLIM, 64);
    if (!mlim) return KDE_ENOMEM;
    spec_mlim_kernel<<<1, 1, 0, ctx->stream>>>(cl, argmin_dev, mlim);
    KDE_LAUNCHED(ctx, "spec_mlim_kernel");
    double2 *S = nullptr;
    KDE_TRY(spec_structure(ctx, u, N, Mmax, mlim, &S));
    return spec_loo_from_S(ctx, u, N, L, S, cl, Mmax, argmin_dev, loo);
}

int kde_spec_modes(double kappa) { return spec_modes(kappa); }

kde_status kde_cv_spectral_device(kde_ctx *ctx, const uint32_t *u, int64_t N, double L, const double *cand_host,
                                  int n_cand, double *cv_dev, int *argmin_dev, float *loo, double *kstar_dev)
{
    CandList cl{};
    cl.n = n_cand;
    cl.scale_mode = 0;
    double kmax = 0.0;
    for (int c = 0; c < n_cand; ++c) {
        cl.k[c] = cand_host[c];
        kmax = cand_host[c] > kmax ? cand_host[c] : kmax;
    }
    const int M = spec_modes(kmax);
    const int Astride = M + 1;
    double *Atab = (double *)kde_ws(ctx, WS_SP_A, (size_t)n_cand * Astride * 8 + 64 * 1024 * 8);
    if (!Atab) return KDE_ENOMEM;
    double2 *S = nullptr;
    KDE_TRY(spec_structure(ctx, u, N, M, nullptr, &S));
    // the Bessel ratios depend on the candidates only: a width schedule that repeats its
    // candidate list reuses the table the previous call left in the workspace
    std::vector<double> key(cand_host, cand_host + n_cand);
    const bool ready = ctx->sp_atab == (void *)Atab && ctx->sp_atab_cands == key;
    spec_cv_kernel<<<n_cand, SP_THREADS, 0, ctx->stream>>>(S, cl, N, L, Astride, Atab, ready ? 1 : 0, cv_dev);
    ctx->sp_atab = (void *)Atab;
    ctx->sp_atab_cands = key;
    KDE_LAUNCHED(ctx, "spec_cv_kernel");
    spec_argmin_kernel<<<1, 1, 0, ctx->stream>>>(cv_dev, cl, argmin_dev, kstar_dev);
    KDE_LAUNCHED(ctx, "spec_argmin_kernel");
    if (loo) KDE_TRY(spec_loo_from_S(ctx, u, N, L, S, cl, M, argmin_dev, loo, Atab, Astride));
    return KDE_OK;
}
