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
// atomics: exact) and, on the way, the slice's total: each lane's partial sum t
// is split into four 16-bit fields whose warp sums (one redux each) cannot
// overflow, and recombined into the sums of t >> 32 and t mod 2^32, which stay
// exact in int64 over the whole grid.  After one cluster barrier every CTA
// gathers every node's sum through distributed shared memory as
// rho'_g = charge acc_inv (n_g - M) with M the grid mean sum_l n_l / Ng to FP32
// precision (the background is a constant and drops out; so does the tiny
// remainder of the mean, which the zero-sum Green's function annihilates), and
// solves the circular convolution for its own slice as poisson_kernel does.  No
// step uses FP64, which is slow on this part.  The second cluster barrier, which
// keeps every CTA's shared memory alive until the others have read it, is split:
// a CTA arrives once its remote reads are done and waits only before it exits.
// Replaces the row reduction, the accumulator round trip and the Poisson launch
// of the step.
// ---------------------------------------------------------------------------
#define FIELD_C 8
#define FIELD_THREADS 1024
#define FIELD_MAXG 1024
#define FIELD_MAXS ((KDE_MAX_NG + FIELD_C - 1) / FIELD_C)

// 4-byte asynchronous copy global -> shared (completes by cp.async.wait_all)
__device__ __forceinline__ void field_copy_async4(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

__global__ void __cluster_dims__(FIELD_C, 1, 1) __launch_bounds__(FIELD_THREADS)
    field_rows_kernel(const long long *__restrict__ rows, const int2 *__restrict__ hdr, int G, int Ng,
                      float scale62, float inv_ng, const float *__restrict__ Gf, float *E)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ int2 sh[FIELD_MAXG];
    __shared__ long long sacc[FIELD_MAXS];
    __shared__ float rt[KDE_MAX_NG];
    __shared__ float gs[KDE_MAX_NG];
    __shared__ long long s_hl[2];  // the slice's sums of t >> 32 and of t mod 2^32
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = FIELD_THREADS / 32;
    constexpr int RB = 20;  // rows of a warp whose loads are in flight together (608 rows: one batch)
    const int q = (int)cluster.block_rank();
    const int a = (int)((int64_t)Ng * q / FIELD_C), b = (int)((int64_t)Ng * (q + 1) / FIELD_C);
    kde_pdl_wait();  // the rows come from the deposit before
    kde_pdl_trigger();
    for (int k = tid; k < G; k += FIELD_THREADS) sh[k] = hdr[k];
    // the Green's function arrives in shared memory while the rows are summed
    for (int g = tid; g < Ng; g += FIELD_THREADS) field_copy_async4(&gs[g], &Gf[g]);
    for (int g = tid; g < b - a; g += FIELD_THREADS) sacc[g] = 0;
    if (tid < 2) s_hl[tid] = 0;
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
            // t = f3 2^48 + f2 2^32 + f1 2^16 + f0 (f3 signed, |f3| < 2^15; the others in
            // [0, 2^16)): 32 lanes' sums of each field fit 32 bits
            const unsigned long long ut = (unsigned long long)t;
            const unsigned int f0 = __reduce_add_sync(0xffffffffu, (unsigned int)(ut & 0xffffu));
            const unsigned int f1 = __reduce_add_sync(0xffffffffu, (unsigned int)((ut >> 16) & 0xffffu));
            const unsigned int f2 = __reduce_add_sync(0xffffffffu, (unsigned int)((ut >> 32) & 0xffffu));
            const int f3 = __reduce_add_sync(0xffffffffu, (int)(t >> 48));
            if (lane == 0) {
                const long long hi = (long long)f2 + (long long)f3 * 65536ll, lo = (long long)f0 + (long long)f1 * 65536ll;
                if (hi) atomicAdd((unsigned long long *)&s_hl[0], (unsigned long long)hi);
                if (lo) atomicAdd((unsigned long long *)&s_hl[1], (unsigned long long)lo);
            }
        }
    }
    cluster.sync();  // every slice and slice sum is ready (the barrier also orders this CTA's atomics)
    // the whole density minus the mean from every CTA's slice; lanes 0 .. C-1 of a warp
    // fetch the CTAs' slice sums, issued together with the node loads, and add them in
    // FP32 in a fixed order; n_g - M is exact in int64 and rounds once to FP32
    for (int g0 = warp * 32; g0 < Ng; g0 += FIELD_THREADS) {
        const int g = g0 + lane;
        long long hi = 0, lo = 0, n = 0;
        if (lane < FIELD_C) {
            const long long *r = cluster.map_shared_rank(s_hl, lane);
            hi = r[0];
            lo = r[1];
        }
        if (g < Ng) {
            // the CTA whose slice [Ng o / C, Ng (o + 1) / C) holds node g (Ng C < 2^31)
            int o = g * FIELD_C / Ng;
            while (o > 0 && Ng * o / FIELD_C > g) --o;
            while (o < FIELD_C - 1 && Ng * (o + 1) / FIELD_C <= g) ++o;
            n = cluster.map_shared_rank(sacc, o)[g - Ng * o / FIELD_C];
        }
        float s = fmaf(__ll2float_rn(hi), 4294967296.f, __ll2float_rn(lo));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const long long mean = __float2ll_rn(s * inv_ng);
        // (n_g - M) charge acc_inv as (n_g - M) 2^-62 (exact) times charge acc_inv 2^62
        if (g < Ng) rt[g] = __ll2float_rn(n - mean) * 0x1p-62f * scale62;
    }
    // this CTA's remote reads are done; it waits for the others' only before it exits
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
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
    __syncwarp();
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

kde_status kde_field_from_rows(kde_ctx *ctx, const long long *rows, const int2 *hdr, int G, int Ng, double L,
                               double acc_inv, double charge, bool fd, float *E_out)
{
    if (G > FIELD_MAXG) return kde_fail(ctx, KDE_ENOTSUP, "field: %d deposit rows exceed %d", G, FIELD_MAXG);
    const float *Gf = (const float *)kde_green_table(ctx, Ng, L, fd, false);
    if (!Gf) return KDE_ENOMEM;
    {
        KdeProfScope _ps(ctx, PROF_POISSON);
        KDE_CUDA(ctx, kde_launch(ctx, true, field_rows_kernel, dim3(FIELD_C), dim3(FIELD_THREADS), 0, rows, hdr, G, Ng,
                                 (float)(charge * acc_inv * 0x1p62), 1.f / (float)Ng, Gf, E_out),
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
