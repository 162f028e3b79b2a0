// field.cu -- periodic Poisson solve and field energy.
//
// The solve is the circular convolution E_j = sum_l G[(j - l) mod Ng] rho'_l
// with the Green's function of ctx.cu (spectral symbol 1/(i k_m), or the
// finite-difference symbol of Sec. III.A); rho' is the total charge density
// with its mean removed in FP64 (G annihilates constants, and removing the
// mean first keeps the FP32 sum free of cancellation).  Ng <= 4096, so the
// whole grid lives in shared memory; each warp owns one output node, its lanes
// take every 32nd term and a shuffle tree adds them (Ng / 8 blocks of 8 warps).
#include "common.cuh"

#define POI_THREADS 256

template <typename T>
__global__ void __launch_bounds__(POI_THREADS)
    poisson_kernel(const T *rho, const long long *acc, double acc_inv, int Ng, double charge, double background,
                   const T *G, T *E)
{
    extern __shared__ __align__(16) unsigned char sm[];
    T *rt = (T *)sm;
    T *Gs = rt + Ng;
    __shared__ double red[POI_THREADS];
    double local = 0.0;
    for (int l = threadIdx.x; l < Ng; l += POI_THREADS) {
        double r = acc ? (double)acc[l] * acc_inv : (double)rho[l];
        local += background + charge * r;
    }
    red[threadIdx.x] = local;
    __syncthreads();
    for (int o = POI_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double mean = red[0] / Ng;
    for (int l = threadIdx.x; l < Ng; l += POI_THREADS) {
        double r = acc ? (double)acc[l] * acc_inv : (double)rho[l];
        rt[l] = (T)(background + charge * r - mean);
        Gs[l] = G[l];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (POI_THREADS / 32) + (threadIdx.x >> 5);
    if (j >= Ng) return;
    T s = 0;
    for (int l = lane; l < Ng; l += 32) {
        const int d = j - l;
        s += Gs[d < 0 ? d + Ng : d] * rt[l];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) E[j] = s;
}

template <typename T>
__global__ void energy_kernel(const T *E, int Ng, double dx, double *out)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int g = threadIdx.x; g < Ng; g += 256) s += (double)E[g] * (double)E[g];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = 0.5 * red[0] * dx;
}

template <typename T>
kde_status kde_poisson_impl(kde_ctx *ctx, const T *rho, const long long *acc, double acc_inv, int Ng, double L,
                            double charge, double background, bool fd, T *E_out)
{
    const T *G = (const T *)kde_green_table(ctx, Ng, L, fd, sizeof(T) == 8);
    if (!G) return KDE_ENOMEM;
    size_t smem = (size_t)2 * Ng * sizeof(T);
    static bool attr[2] = {false, false};
    if (!attr[sizeof(T) == 8]) {
        cudaFuncSetAttribute(poisson_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             2 * KDE_MAX_NG * (int)sizeof(T));
        attr[sizeof(T) == 8] = true;
    }
    {
        KdeProfScope _ps(ctx, PROF_POISSON);
    poisson_kernel<T><<<(Ng + POI_THREADS / 32 - 1) / (POI_THREADS / 32), POI_THREADS, smem, ctx->stream>>>(
        rho, acc, acc_inv, Ng, charge, background, G, E_out);
    }
    KDE_LAUNCHED(ctx, "poisson_kernel");
    return KDE_OK;
}

template <typename T>
kde_status kde_energy_impl(kde_ctx *ctx, const T *E, int Ng, double L, double *energy_out)
{
    energy_kernel<T><<<1, 256, 0, ctx->stream>>>(E, Ng, L / Ng, energy_out);
    KDE_LAUNCHED(ctx, "energy_kernel");
    return KDE_OK;
}

template kde_status kde_poisson_impl<float>(kde_ctx *, const float *, const long long *, double, int, double, double,
                                            double, bool, float *);
template kde_status kde_poisson_impl<double>(kde_ctx *, const double *, const long long *, double, int, double,
                                             double, double, bool, double *);
template kde_status kde_energy_impl<float>(kde_ctx *, const float *, int, double, double *);
template kde_status kde_energy_impl<double>(kde_ctx *, const double *, int, double, double *);

extern "C" kde_status kde_poisson(kde_ctx *ctx, const void *rho, int32_t Ng, double L, double charge,
                                  double background, void *E_out, double *energy_out, uint32_t flags)
{
    if (!ctx) return KDE_EINVAL;
    if (Ng < 1 || Ng > KDE_MAX_NG || !(L > 0) || !rho || !E_out || rho == E_out)
        return kde_fail(ctx, KDE_EINVAL, "kde_poisson: need 1 <= Ng <= %d, L > 0, distinct non-null arrays",
                        KDE_MAX_NG);
    if (flags & ~(KDE_F64 | KDE_POISSON_FD))
        return kde_fail(ctx, KDE_ENOTSUP, "kde_poisson: unsupported flags 0x%x", flags);
    cudaSetDevice(ctx->device);
    bool fd = (flags & KDE_POISSON_FD) != 0;
    if (flags & KDE_F64) {
        KDE_TRY(kde_poisson_impl<double>(ctx, (const double *)rho, nullptr, 0.0, Ng, L, charge, background, fd,
                                         (double *)E_out));
        if (energy_out) KDE_TRY(kde_energy_impl<double>(ctx, (const double *)E_out, Ng, L, energy_out));
    } else {
        KDE_TRY(kde_poisson_impl<float>(ctx, (const float *)rho, nullptr, 0.0, Ng, L, charge, background, fd,
                                        (float *)E_out));
        if (energy_out) KDE_TRY(kde_energy_impl<float>(ctx, (const float *)E_out, Ng, L, energy_out));
    }
    return KDE_OK;
}
