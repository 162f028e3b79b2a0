// field.cu -- periodic Poisson solve and field energy.
//
// The solve is the circular convolution E_j = sum_l G[(j - l) mod Ng] rho'_l
// with the Green's function of ctx.cu (spectral symbol 1/(i k_m), or the
// finite-difference symbol of Sec. III.A); rho' is the total charge density
// with its mean removed in FP64 (G annihilates constants, and removing the
// mean first keeps the FP32 sum free of cancellation).  Ng <= 4096, so the
// whole grid lives in shared memory; each warp owns one output node, its lanes
// take every 32nd term and a shuffle tree adds them (Ng / 8 blocks of 8 warps).
#include <cooperative_groups.h>

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

// ---------------------------------------------------------------------------
// Field of the PIC step straight from the FP32 deposit's per-CTA rows: one
// cluster of FIELD_C CTAs.  CTA q owns the node slice [q Ng / C, (q + 1) Ng / C):
// its warps take the rows in turn (headers staged in shared memory), add every
// row entry that falls in the slice into the slice's int64 sums (shared-memory
// atomics: exact).  Each CTA converts its slice to the total charge density in
// FP64 and sums it; after one cluster barrier every CTA adds the slice sums in rank
// order (the same mean in every CTA), gathers every slice minus the mean through
// distributed shared memory and solves the circular convolution for its own slice
// as poisson_kernel does.  Replaces the row reduction, the accumulator round trip and
// the Poisson launch of the step.
// ---------------------------------------------------------------------------
#define FIELD_C 8
#define FIELD_THREADS 1024
#define FIELD_MAXG 1024
#define FIELD_MAXS ((KDE_MAX_NG + FIELD_C - 1) / FIELD_C)

__global__ void __cluster_dims__(FIELD_C, 1, 1) __launch_bounds__(FIELD_THREADS)
    field_rows_kernel(const long long *__restrict__ rows, const int2 *__restrict__ hdr, int G, int Ng, double acc_inv,
                      double charge, double background, const float *__restrict__ Gf, float *E)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ int2 sh[FIELD_MAXG];
    __shared__ long long sacc[FIELD_MAXS];
    __shared__ float rt[KDE_MAX_NG];
    __shared__ float gs[KDE_MAX_NG];
    __shared__ double red[FIELD_THREADS / 32];
    __shared__ double s_psum, s_mean;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = FIELD_THREADS / 32;
    constexpr int RB = 20;  // rows of a warp whose loads are in flight together (608 rows: one batch)
    const int q = (int)cluster.block_rank();
    const int a = (int)((int64_t)Ng * q / FIELD_C), b = (int)((int64_t)Ng * (q + 1) / FIELD_C);
    kde_pdl_wait();  // the rows come from the deposit before
    kde_pdl_trigger();
    for (int k = tid; k < G; k += FIELD_THREADS) sh[k] = hdr[k];
    for (int g = tid; g < Ng; g += FIELD_THREADS) gs[g] = Gf[g];  // used after the row sums
    for (int g = tid; g < b - a; g += FIELD_THREADS) sacc[g] = 0;
    __syncthreads();
    // rows of warp w: w, w + 32, ...; for each row the slice nodes its window covers
    for (int k0 = warp; k0 < G; k0 += RB * NW) {
        for (int g0 = a; g0 < b; g0 += 32) {
            const int g = g0 + lane;
            long long v[RB];
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                const int k = k0 + i * NW;
                v[i] = 0;
                if (k < G && g < b) {
                    const int2 h = sh[k];
                    int r = g - h.x;
                    r = r < 0 ? r + Ng : (r >= Ng ? r - Ng : r);
                    if (r < h.y) v[i] = rows[(size_t)k * Ng + r];
                }
            }
            long long t = 0;
#pragma unroll
            for (int i = 0; i < RB; ++i) t += v[i];
            if (t) atomicAdd((unsigned long long *)&sacc[g - a], (unsigned long long)t);
        }
    }
    __syncthreads();
    // the slice's total charge density in FP64, in place of its integer sums (the other
    // CTAs read it there), and its sum: one value a thread, warp sums, the block sum in
    // warp order on one warp (FP64 is slow on this part)
    double *dsl = (double *)sacc;
    double local = 0.0;
    for (int g = tid; g < b - a; g += FIELD_THREADS) {
        const double t = background + charge * ((double)sacc[g] * acc_inv);
        dsl[g] = t;
        local += t;
    }
    if (warp * 32 < b - a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    }
    if (lane == 0) red[warp] = local;
    __syncthreads();
    if (warp == 0) {
        double v = red[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_psum = v;
    }
    cluster.sync();  // every slice and slice sum is ready
    if (warp == 0) {
        // the mean from the slice sums in rank order: the same value in every CTA
        const double p = lane < FIELD_C ? *cluster.map_shared_rank(&s_psum, lane) : 0.0;
        double m = 0.0;
#pragma unroll
        for (int o = 0; o < FIELD_C; ++o) m += __shfl_sync(0xffffffffu, p, o);
        if (lane == 0) s_mean = m / Ng;
    }
    __syncthreads();
    const double mean = s_mean;
    // the whole density minus the mean from every CTA's slice
    for (int g = tid; g < Ng; g += FIELD_THREADS) {
        // the CTA whose slice [Ng o / C, Ng (o + 1) / C) holds node g (Ng C < 2^31)
        int o = g * FIELD_C / Ng;
        while (o > 0 && Ng * o / FIELD_C > g) --o;
        while (o < FIELD_C - 1 && Ng * (o + 1) / FIELD_C <= g) ++o;
        rt[g] = (float)(cluster.map_shared_rank(dsl, o)[g - Ng * o / FIELD_C] - mean);
    }
    cluster.sync();  // every remote read is done before any CTA moves on (and may exit)
    // E_j = sum_l G[(j - l) mod Ng] rho'_l for the slice: one node a warp at a time
    for (int j = a + warp; j < b; j += NW) {
        float s2 = 0.f;
        for (int l = lane; l < Ng; l += 32) {
            const int d = j - l;
            s2 += gs[d < 0 ? d + Ng : d] * rt[l];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if (lane == 0) E[j] = s2;
    }
}

kde_status kde_field_from_rows(kde_ctx *ctx, const long long *rows, const int2 *hdr, int G, int Ng, double L,
                               double acc_inv, double charge, double background, bool fd, float *E_out)
{
    if (G > FIELD_MAXG) return kde_fail(ctx, KDE_ENOTSUP, "field: %d deposit rows exceed %d", G, FIELD_MAXG);
    const float *Gf = (const float *)kde_green_table(ctx, Ng, L, fd, false);
    if (!Gf) return KDE_ENOMEM;
    {
        KdeProfScope _ps(ctx, PROF_POISSON);
        KDE_CUDA(ctx, kde_launch(ctx, true, field_rows_kernel, dim3(FIELD_C), dim3(FIELD_THREADS), 0, rows, hdr, G, Ng,
                                 acc_inv, charge, background, Gf, E_out),
                 "field_rows_kernel");
    }
    KDE_LAUNCHED(ctx, "field_rows_kernel");
    return KDE_OK;
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
