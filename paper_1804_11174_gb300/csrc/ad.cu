// ad.cu -- Anderson-Darling test of the particle positions against the
// uniform distribution on the domain (Sec. II.D), the statistic that drives
// the width-update algorithm.
//
// Sample values are the position codes' cell centres, F_i = (u_i + 1/2) / 2^32.
// With the codes sorted ascending (LSD radix sort) and j the 1-based rank,
//   A^2 = -n - (1/n) S,  S = sum_j (2j - 1) ln F_(j) + (2n + 1 - 2j) ln(1 - F_(j)),
// which is the textbook sum with the second logarithm re-indexed.  S is O(n^2)
// while A^2 is O(1), so S is accumulated in FP64, and FP64 operations (slow on
// this GPU) are kept off the per-sample path: per 2^16-code bin b with first
// code u_b, for a sample d = u - u_b codes into the bin,
//   ln F = ln F_b + d r1 + c(d r1),   ln(1 - F) = ln(1 - F_b) - d r2 + c(-d r2),
// r1 = 1 / (u_b + 1/2), r2 = 1 / (2^32 - u_b - 1/2), c(x) = log1p(x) - x.  Over a
// run of samples in one bin the weighted sums of 1 and of d are exact integers,
// so the FP64 part (table values ln F_b, ln(1 - F_b), r1, r2) is applied once
// per run; the small remainder c(x) = x^2 (-1/2 + x/3 - x^2/4 + x^3/5) (|x| <
// 2^-8, Taylor series of log1p, truncation below 2^-48) is summed in FP32.
// In the first and last 256 bins, where x is not small, the logarithm that is
// affected is taken in FP64 per sample.  The partition of the sorted array
// into blocks depends only on n and every sum runs in a fixed order: the
// result is bitwise reproducible.
//
// p-value: Marsaglia & Marsaglia (2004), "Evaluating the Anderson-Darling
// distribution" (J. Stat. Softw. 9(2)): the limiting distribution by their two
// fitted expressions plus their finite-n correction, up to A^2 = 7; beyond, the
// large-A^2 law of the limiting distribution, P ~ C (A^2)^{-1/2} e^{-A^2} (the
// first chi^2 term of A^2 = sum_j chi^2_1 / (j (j + 1)) dominates), with C from
// the value at 7.  Returned as ln p, which does not underflow.
#include "common.cuh"

#define AD_BITS 16                    // table bins: the top 16 bits of the code
#define AD_NBINS (1 << AD_BITS)
#define AD_EDGE 256                   // bins at each end taken in FP64 per sample
#define AD_THREADS 128
#define AD_PER 16                     // consecutive sorted samples per thread
#define AD_TILE (AD_THREADS * AD_PER)  // samples per block
#define AD_ZJOIN 7.0

struct AdBin {
    double lnF, ln1mF;  // ln F_b, ln(1 - F_b) at the bin's first code
    double r1, r2;      // 1 / (u_b + 1/2), 1 / (2^32 - u_b - 1/2)
    float r1f, r2f;     // the same in FP32
};

__global__ void ad_table_kernel(AdBin *tab)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= AD_NBINS) return;
    const double c = (double)b * 65536.0 + 0.5;  // u_b + 1/2
    AdBin t;
    t.lnF = log(c * (1.0 / 4294967296.0));
    t.ln1mF = log1p(-c * (1.0 / 4294967296.0));
    t.r1 = 1.0 / c;
    t.r2 = 1.0 / (4294967296.0 - c);
    t.r1f = (float)t.r1;
    t.r2f = (float)t.r2;
    tab[b] = t;
}

// log1p(x) - x for |x| < 2^-8
__device__ __forceinline__ float ad_log1p_rem(float x)
{
    return x * x * fmaf(x, fmaf(x, fmaf(x, 0.2f, -0.25f), 1.0f / 3.0f), -0.5f);
}

// one block per AD_TILE sorted samples; thread t takes samples base + t*AD_PER + q
__global__ void __launch_bounds__(AD_THREADS)
    ad_terms_kernel(const uint32_t *__restrict__ z, int64_t N, const AdBin *__restrict__ tab, double *part)
{
    __shared__ double red[AD_THREADS];
    const int64_t i0 = (int64_t)blockIdx.x * AD_TILE + (int64_t)threadIdx.x * AD_PER;
    double big = 0.0;
    float small = 0.f;
    int cur = -1;
    // over the current bin run: sums of the weights wa = 2j - 1, wb = 2n + 1 - 2j
    // and of wa d, wb d (exact integers)
    long long sa = 0, sb = 0, sad = 0, sbd = 0;
    AdBin tb{};
    auto flush = [&]() { big += (double)sa * tb.lnF + (double)sad * tb.r1 + (double)sb * tb.ln1mF - (double)sbd * tb.r2; };
#pragma unroll 4
    for (int q = 0; q < AD_PER; ++q) {
        const int64_t i = i0 + q;
        if (i >= N) break;
        const uint32_t y = z[i];
        const int b = (int)(y >> AD_BITS);
        const long long d = (long long)(y & (AD_NBINS - 1));
        if (b != cur) {
            if (cur >= 0) flush();
            sa = sb = sad = sbd = 0;
            cur = b;
            tb = tab[b];
        }
        const long long wa = 2 * (i + 1) - 1, wb = 2 * N + 1 - 2 * (i + 1);
        if (b < AD_EDGE) {
            big += (double)wa * log(((double)y + 0.5) * (1.0 / 4294967296.0));
        } else {
            sa += wa;
            sad += wa * d;
            small = fmaf((float)wa, ad_log1p_rem((float)d * tb.r1f), small);
        }
        if (b >= AD_NBINS - AD_EDGE) {
            big += (double)wb * log1p(-((double)y + 0.5) * (1.0 / 4294967296.0));
        } else {
            sb += wb;
            sbd += wb * d;
            small = fmaf((float)wb, ad_log1p_rem(-(float)d * tb.r2f), small);
        }
    }
    if (cur >= 0) flush();
    red[threadIdx.x] = big + (double)small;
    __syncthreads();
    for (int o = AD_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Marsaglia & Marsaglia: limiting distribution function, two fitted expressions
__device__ double ad_limit_cdf(double z)
{
    if (z <= 0.0) return 0.0;
    if (z < 2.0)
        return exp(-1.2337141 / z) / sqrt(z) *
               (2.00012 + (0.247105 - (0.0649821 - (0.0347962 - (0.011672 - 0.00168691 * z) * z) * z) * z) * z);
    return exp(-exp(1.0776 - (2.30695 - (0.43424 - (0.082433 - (0.008056 - 0.0003146 * z) * z) * z) * z) * z));
}

// their finite-n correction as a function of n and the limiting value x
__device__ double ad_finite_n(double n, double x)
{
    if (x > 0.8)
        return (-130.2137 + (745.2337 - (1705.091 - (1950.646 - (1116.360 - 255.7844 * x) * x) * x) * x) * x) / n;
    const double c = 0.01265 + 0.1757 / n;
    if (x < c) {
        double t = x / c;
        t = sqrt(t) * (1.0 - t) * (49.0 * t - 102.0);
        return t * (0.0037 / (n * n) + 0.00078 / n + 0.00006) / n;
    }
    double t = (x - c) / (0.8 - c);
    t = -0.00022633 + (6.54034 - (14.6538 - (14.458 - (8.259 - 1.91864 * t) * t) * t) * t) * t;
    return t * (0.04213 + 0.01365 / n) / n;
}

__device__ double ad_cdf(double z, double n)
{
    const double x = ad_limit_cdf(z);
    const double p = x + ad_finite_n(n, x);
    return p < 0.0 ? 0.0 : (p > 1.0 ? 1.0 : p);
}

__device__ double ad_log_pvalue(double a2, double n)
{
    if (a2 <= AD_ZJOIN) return log(1.0 - ad_cdf(a2, n));
    return log(1.0 - ad_cdf(AD_ZJOIN, n)) + 0.5 * log(AD_ZJOIN / a2) + (AD_ZJOIN - a2);
}

// S over the block partials in block order, then A^2 and ln p
__global__ void __launch_bounds__(1024) ad_final_kernel(const double *part, int nparts, int64_t N, double *out,
                                                        double *lp_slot)
{
    __shared__ double red[1024];
    double s = 0.0;
    for (int k = threadIdx.x; k < nparts; k += 1024) s += part[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double n = (double)N;
        const double a2 = -n - red[0] / n;
        const double lp = ad_log_pvalue(a2, n);
        out[0] = a2;
        out[1] = lp;
        if (lp_slot) *lp_slot = lp;
    }
}

static const AdBin *ad_table(kde_ctx *ctx)
{
    if (ctx->ad_tab) return (const AdBin *)ctx->ad_tab;
    void *p = nullptr;
    if (cudaMalloc(&p, sizeof(AdBin) * AD_NBINS) != cudaSuccess) {
        cudaGetLastError();
        kde_fail(ctx, KDE_ENOMEM, "Anderson-Darling table allocation failed");
        return nullptr;
    }
    ad_table_kernel<<<AD_NBINS / 256, 256, 0, ctx->stream>>>((AdBin *)p);
    if (cudaGetLastError() != cudaSuccess) {
        cudaFree(p);
        kde_fail(ctx, KDE_ECUDA, "Anderson-Darling table kernel launch failed");
        return nullptr;
    }
    ++ctx->launches;
    ctx->ad_tab = p;
    return (const AdBin *)p;
}

kde_status kde_ad_device(kde_ctx *ctx, const uint32_t *u, int64_t N, double *out_dev, double *lp_slot)
{
    const AdBin *tab = ad_table(ctx);
    if (!tab) return KDE_ENOMEM;
    const int nparts = (int)((N + AD_TILE - 1) / AD_TILE);
    uint32_t *z = (uint32_t *)kde_ws(ctx, WS_AD_Z, (size_t)N * 4);
    uint32_t *t = (uint32_t *)kde_ws(ctx, WS_AD_T, (size_t)N * 4);
    double *part = (double *)kde_ws(ctx, WS_AD_PART, (size_t)nparts * 8);
    if (!z || !t || !part) return KDE_ENOMEM;
    KDE_TRY(kde_radix_sort_u32(ctx, u, N, z, t));
    {
        KdeProfScope _ps(ctx, PROF_AD);
        ad_terms_kernel<<<nparts, AD_THREADS, 0, ctx->stream>>>(z, N, tab, part);
    }
    KDE_LAUNCHED(ctx, "ad_terms_kernel");
    ad_final_kernel<<<1, 1024, 0, ctx->stream>>>(part, nparts, N, out_dev, lp_slot);
    KDE_LAUNCHED(ctx, "ad_final_kernel");
    return KDE_OK;
}

extern "C" kde_status kde_ad_test(kde_ctx *ctx, const uint32_t *u, int64_t N, double *a2_out, double *log_p_out)
{
    if (!ctx) return KDE_EINVAL;
    if (N < KDE_AD_MIN_N || N > 0xFFFFFFFFll || !u)
        return kde_fail(ctx, KDE_EINVAL, "kde_ad_test: need %d <= N < 2^32 and a position array", KDE_AD_MIN_N);
    cudaSetDevice(ctx->device);
    double *out = (double *)kde_ws(ctx, WS_AD_OUT, 16);
    if (!out) return KDE_ENOMEM;
    KDE_TRY(kde_ad_device(ctx, u, N, out, nullptr));
    double h[2];
    KDE_CUDA(ctx, cudaMemcpyAsync(h, out, 16, cudaMemcpyDeviceToHost, ctx->stream), "AD result copy");
    KDE_TRY(kde_sync(ctx));
    if (a2_out) *a2_out = h[0];
    if (log_p_out) *log_p_out = h[1];
    return KDE_OK;
}
