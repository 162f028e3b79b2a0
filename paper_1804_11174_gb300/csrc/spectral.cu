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
// arithmetic, then one FP32 sincospi.  Sub-chunk sums run in FP32 and are
// combined in FP64 in a fixed order; the CV combination and the leave-one-out
// sums are FP64.  Particles may come in any order (no sort).
#include "common.cuh"

#define SP_THREADS 256
#define SP_SUB 256
#define SP_MAXM 16384
#define SP_MAXCHUNK 16384

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

// structure factor partials: block (chunk, mode block); thread = one mode
__global__ void __launch_bounds__(SP_THREADS)
    spec_sf_kernel(const uint32_t *__restrict__ u, int64_t N, int64_t chunk, int M, double2 *part)
{
    extern __shared__ uint32_t us[];
    const int64_t j0 = (int64_t)blockIdx.x * chunk;
    const int n = (int)(N - j0 < chunk ? N - j0 : chunk);
    for (int k = threadIdx.x; k < n; k += SP_THREADS) us[k] = u[j0 + k];
    __syncthreads();
    const int m = 1 + blockIdx.y * SP_THREADS + threadIdx.x;
    if (m > M) return;
    double cr = 0.0, ci = 0.0;
    for (int k0 = 0; k0 < n; k0 += SP_SUB) {
        const int k1 = k0 + SP_SUB < n ? k0 + SP_SUB : n;
        float fr = 0.f, fi = 0.f;
#pragma unroll 4
        for (int k = k0; k < k1; ++k) {
            const uint32_t ph = (uint32_t)m * us[k];  // m theta / (2 pi) in 2^-32 turns
            float s, c;
            sincospif((float)(int32_t)ph * (1.0f / 2147483648.0f), &s, &c);
            fr += c;
            fi += s;
        }
        cr += (double)fr;
        ci += (double)fi;
    }
    part[(size_t)blockIdx.x * M + (m - 1)] = make_double2(cr, ci);
}

// S_m = sum over chunks in chunk order
__global__ void spec_reduce_kernel(const double2 *part, int nchunks, int M, double2 *S)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double sr = 0.0, si = 0.0;
    for (int c = 0; c < nchunks; ++c) {
        double2 p = part[(size_t)c * M + m];
        sr += p.x;
        si += p.y;
    }
    S[m] = make_double2(sr, si);
}

// per candidate (caller's order): Bessel ratios, the three mode sums and CV (x
// units); then argmin (smallest index on ties) and the selected width
__global__ void spec_cv_kernel(const double2 *S, CandList cl, int64_t N, double L, int Astride, double *Atab,
                               double *cv_out, int *argmin, double *kstar)
{
    const int c = threadIdx.x;
    const double n = (double)N;
    if (c < cl.n) {
        const double kappa = cl.k[c];
        const int M = spec_modes(kappa);
        double *A = Atab + (size_t)c * Astride;
        spec_ratios(kappa, M, A);
        double sA = 0.0, sAS = 0.0, sA2S = 0.0;
        for (int m = 1; m <= M; ++m) {
            const double2 s = S[m - 1];
            const double p = s.x * s.x + s.y * s.y;
            sA += A[m];
            sAS += A[m] * p;
            sA2S += A[m] * A[m] * p;
        }
        const double f2 = (n * n + 2.0 * sA2S) / (KDE_TWO_PI * n * n);
        const double pairs = (n * n + 2.0 * sAS - n - 2.0 * n * sA) / KDE_TWO_PI;
        cv_out[c] = (KDE_TWO_PI / L) * (f2 - 2.0 * pairs / (n * (n - 1.0)));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int best = 0;
        for (int q = 1; q < cl.n; ++q)
            if (cv_out[q] < cv_out[best]) best = q;
        *argmin = best;
        if (kstar) *kstar = cl.k[best];
    }
}

// leave-one-out density at the selected width for every particle (input order)
__global__ void __launch_bounds__(SP_THREADS)
    spec_loo_kernel(const uint32_t *__restrict__ u, int64_t N, const double2 *S, CandList cl, int Astride,
                    const double *Atab, const int *argmin, double xs, float *loo)
{
    __shared__ double sA[512];
    __shared__ double2 sS[512];
    const int c = *argmin;
    const double kappa = cl.k[c];
    const int M = spec_modes(kappa);
    const double *A = Atab + (size_t)c * Astride;
    const int64_t i = (int64_t)blockIdx.x * SP_THREADS + threadIdx.x;
    const uint32_t ui = i < N ? u[i] : 0u;
    double acc = 0.0;
    for (int m0 = 1; m0 <= M; m0 += 512) {
        const int cnt = M - m0 + 1 < 512 ? M - m0 + 1 : 512;
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += SP_THREADS) {
            sA[k] = A[m0 + k];
            sS[k] = S[m0 + k - 1];
        }
        __syncthreads();
        for (int k = 0; k < cnt; ++k) {
            const uint32_t ph = (uint32_t)(m0 + k) * ui;
            float s, co;
            sincospif((float)(int32_t)ph * (1.0f / 2147483648.0f), &s, &co);
            const double2 q = sS[k];
            // Re(e^{i m theta_i} conj(S_m)) = cos * Sr + sin * Si
            acc += sA[k] * ((double)co * q.x + (double)s * q.y);
        }
    }
    if (i >= N) return;
    const double n = (double)N;
    const double all = (n + 2.0 * acc) / KDE_TWO_PI;
    loo[i] = (float)(xs * (all - kde_norm(kappa)) / (n - 1.0));
}

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
    int64_t chunk = 4096;
    while ((N + chunk - 1) / chunk > 256 && chunk < SP_MAXCHUNK) chunk *= 2;
    const int nchunks = (int)((N + chunk - 1) / chunk);
    const int Astride = M + 1;
    double2 *part = (double2 *)kde_ws(ctx, WS_SP_PART, (size_t)nchunks * M * sizeof(double2));
    double2 *S = (double2 *)kde_ws(ctx, WS_SP_S, (size_t)M * sizeof(double2));
    double *Atab = (double *)kde_ws(ctx, WS_SP_A, (size_t)n_cand * Astride * 8 + 64 * 1024 * 8);
    if (!part || !S || !Atab) return KDE_ENOMEM;
    static bool attr = false;
    if (!attr) {
        KDE_CUDA(ctx, cudaFuncSetAttribute(spec_sf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           SP_MAXCHUNK * 4),
                 "spec_sf_kernel attribute");
        attr = true;
    }
    const size_t smem = (size_t)chunk * 4;
    {
        KdeProfScope _ps(ctx, PROF_SPECTRAL);
        dim3 grid((unsigned)nchunks, (unsigned)((M + SP_THREADS - 1) / SP_THREADS));
        spec_sf_kernel<<<grid, SP_THREADS, smem, ctx->stream>>>(u, N, chunk, M, part);
    }
    KDE_LAUNCHED(ctx, "spec_sf_kernel");
    spec_reduce_kernel<<<(M + 255) / 256, 256, 0, ctx->stream>>>(part, nchunks, M, S);
    KDE_LAUNCHED(ctx, "spec_reduce_kernel");
    spec_cv_kernel<<<1, 256, 0, ctx->stream>>>(S, cl, N, L, Astride, Atab, cv_dev, argmin_dev, kstar_dev);
    KDE_LAUNCHED(ctx, "spec_cv_kernel");
    if (loo) {
        spec_loo_kernel<<<(unsigned)((N + SP_THREADS - 1) / SP_THREADS), SP_THREADS, 0, ctx->stream>>>(
            u, N, S, cl, Astride, Atab, argmin_dev, KDE_TWO_PI / L, loo);
        KDE_LAUNCHED(ctx, "spec_loo_kernel");
    }
    return KDE_OK;
}
