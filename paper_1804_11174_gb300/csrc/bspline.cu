// bspline.cu -- standard-PIC particle shapes for the comparison of Sec. IV
// (Fig. compare_high_order): centred cardinal B-splines of degree P = 1 (CIC),
// 2, 3 and 5, scaled to a width h, S(x) = (1/h) B_P(x/h) with support (P+1) h;
// h = dx gives the standard PIC shape.
//
// Deposit: one thread per particle adds its few node weights into a per-CTA
// shared-memory grid of int64 fixed-point accumulators (exact, so the sum does
// not depend on the order), and each CTA then adds its grid to the global one.
// Gather: one thread per particle, the field staged in shared memory.  Node
// offsets come from the exact integer product u Ng (cell and fraction).
#include "common.cuh"

#define BSP_THREADS 256

// centred cardinal B-splines, written on the distance to the support's edge
// where the polynomial pieces would otherwise cancel
template <int P>
__device__ __forceinline__ float bsp_eval(float t)
{
    const float a = fabsf(t);
    if (P == 1) return fmaxf(0.f, 1.f - a);
    if (P == 2) {
        if (a <= 0.5f) return 0.75f - a * a;
        if (a < 1.5f) {
            const float b = 1.5f - a;
            return 0.5f * b * b;
        }
        return 0.f;
    }
    if (P == 3) {
        if (a < 2.f) {
            const float b = 2.f - a, c = 1.f - a;
            const float v = b * b * b;
            return (a <= 1.f ? v - 4.f * c * c * c : v) * (1.f / 6.f);
        }
        return 0.f;
    }
    // P == 5
    if (a <= 1.f) {
        const float a2 = a * a;
        return 0.55f + a2 * (-0.5f + a2 * (0.25f - a * (1.f / 12.f)));
    }
    if (a < 3.f) {
        const float b = 3.f - a, b2 = b * b, v = b2 * b2 * b;
        if (a <= 2.f) {
            const float c = 2.f - a, c2 = c * c;
            return (v - 6.f * c2 * c2 * c) * (1.f / 120.f);
        }
        return v * (1.f / 120.f);
    }
    return 0.f;
}

template <int P>
__global__ void __launch_bounds__(BSP_THREADS)
    bsp_deposit_kernel(const uint32_t *__restrict__ u, int64_t N, int Ng, float r, int W, float wcoef, double scale,
                       long long *acc)
{
    extern __shared__ long long sg[];
    for (int g = threadIdx.x; g < Ng; g += BSP_THREADS) sg[g] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * BSP_THREADS + threadIdx.x; i < N; i += (int64_t)gridDim.x * BSP_THREADS) {
        const uint64_t q = (uint64_t)u[i] * (uint64_t)Ng;
        const int cell = (int)(q >> 32);
        const float frac = (float)(uint32_t)q * (1.0f / 4294967296.0f);
        for (int k = -W; k <= W; ++k) {
            const float b = bsp_eval<P>(((float)k - frac) * r);
            if (b > 0.f) {
                int g = (cell + k) % Ng;
                g = g < 0 ? g + Ng : g;
                const long long v = __double2ll_rn((double)(b * wcoef) * scale);
                if (v) atomicAdd((unsigned long long *)&sg[g], (unsigned long long)v);
            }
        }
    }
    __syncthreads();
    for (int g = threadIdx.x; g < Ng; g += BSP_THREADS)
        if (sg[g]) atomicAdd((unsigned long long *)&acc[g], (unsigned long long)sg[g]);
}

template <int P>
__global__ void __launch_bounds__(BSP_THREADS)
    bsp_gather_kernel(const uint32_t *__restrict__ u, int64_t N, int Ng, float r, int W, const float *__restrict__ field,
                      float *out)
{
    extern __shared__ float sf[];
    for (int g = threadIdx.x; g < Ng; g += BSP_THREADS) sf[g] = field[g];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * BSP_THREADS + threadIdx.x; i < N; i += (int64_t)gridDim.x * BSP_THREADS) {
        const uint64_t q = (uint64_t)u[i] * (uint64_t)Ng;
        const int cell = (int)(q >> 32);
        const float frac = (float)(uint32_t)q * (1.0f / 4294967296.0f);
        float e = 0.f;
        for (int k = -W; k <= W; ++k) {
            const float b = bsp_eval<P>(((float)k - frac) * r);
            int g = (cell + k) % Ng;
            g = g < 0 ? g + Ng : g;
            e = fmaf(b, sf[g], e);
        }
        out[i] = e * r;  // dx / h
    }
}

static double bsp_peak(int P)
{
    return P == 1 ? 1.0 : P == 2 ? 0.75 : P == 3 ? 2.0 / 3.0 : 0.55;
}

// node half-window: |g - s| < (P+1)/2 h/dx, one node of margin
static int bsp_window(int P, double h, double dx) { return (int)ceil(0.5 * (P + 1) * h / dx) + 1; }

static kde_status bsp_check(kde_ctx *ctx, const char *what, const uint32_t *u, int64_t N, int order, double h, int Ng,
                            double L)
{
    if (!ctx) return KDE_EINVAL;
    if (N < 0 || N > 0xFFFFFFFFll || (N > 0 && !u) || Ng < 1 || Ng > KDE_MAX_NG || !(L > 0) ||
        !(order == 1 || order == 2 || order == 3 || order == 5) || !(h > 0) || !((order + 1) * h < L))
        return kde_fail(ctx, KDE_EINVAL,
                        "%s: need 0 <= N < 2^32, 1 <= Ng <= %d, L > 0, order in {1, 2, 3, 5} and 0 < (order+1) h < L",
                        what, KDE_MAX_NG);
    return KDE_OK;
}

static int bsp_grid(kde_ctx *ctx, int64_t N)
{
    int64_t g = (N + BSP_THREADS - 1) / BSP_THREADS;
    const int64_t cap = (int64_t)ctx->sm_count * 8;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

extern "C" kde_status kde_deposit_bspline(kde_ctx *ctx, const uint32_t *u, int64_t N, int32_t order, double h,
                                          int32_t Ng, double L, float *rho_out)
{
    KDE_TRY(bsp_check(ctx, "kde_deposit_bspline", u, N, order, h, Ng, L));
    if (!rho_out) return kde_fail(ctx, KDE_EINVAL, "kde_deposit_bspline: null output");
    cudaSetDevice(ctx->device);
    long long *acc = (long long *)kde_ws(ctx, WS_ACC, (size_t)Ng * 8);
    if (!acc) return KDE_ENOMEM;
    KDE_CUDA(ctx, cudaMemsetAsync(acc, 0, (size_t)Ng * 8, ctx->stream), "bspline acc memset");
    const double dx = L / Ng;
    const float r = (float)(dx / h);
    const int W = bsp_window(order, h, dx);
    const double wcoef = (L / (double)(N > 0 ? N : 1)) / h;  // w_i / h with w_i = L/N
    const double bound = (double)N * wcoef * bsp_peak(order) * 1.0000001 + 1e-300;
    const double scale = kde_acc_scale(bound);
    if (N > 0) {
        const int grid = bsp_grid(ctx, N);
        const size_t smem = (size_t)Ng * 8;
        KdeProfScope _ps(ctx, PROF_DEPOSIT);
        switch (order) {
        case 1: bsp_deposit_kernel<1><<<grid, BSP_THREADS, smem, ctx->stream>>>(u, N, Ng, r, W, (float)wcoef, scale, acc); break;
        case 2: bsp_deposit_kernel<2><<<grid, BSP_THREADS, smem, ctx->stream>>>(u, N, Ng, r, W, (float)wcoef, scale, acc); break;
        case 3: bsp_deposit_kernel<3><<<grid, BSP_THREADS, smem, ctx->stream>>>(u, N, Ng, r, W, (float)wcoef, scale, acc); break;
        default: bsp_deposit_kernel<5><<<grid, BSP_THREADS, smem, ctx->stream>>>(u, N, Ng, r, W, (float)wcoef, scale, acc); break;
        }
    }
    KDE_LAUNCHED(ctx, "bsp_deposit_kernel");
    return kde_acc_to_real<float>(ctx, acc, Ng, bound, nullptr, 0.0, rho_out);
}

extern "C" kde_status kde_gather_bspline(kde_ctx *ctx, const uint32_t *u, int64_t N, int32_t order, double h,
                                         const float *field, int32_t Ng, double L, float *out)
{
    KDE_TRY(bsp_check(ctx, "kde_gather_bspline", u, N, order, h, Ng, L));
    if (!field || (N > 0 && !out)) return kde_fail(ctx, KDE_EINVAL, "kde_gather_bspline: null field or output");
    if (N == 0) return KDE_OK;
    cudaSetDevice(ctx->device);
    const double dx = L / Ng;
    const float r = (float)(dx / h);
    const int W = bsp_window(order, h, dx);
    const int grid = bsp_grid(ctx, N);
    const size_t smem = (size_t)Ng * 4;
    {
        KdeProfScope _ps(ctx, PROF_GATHER);
        switch (order) {
        case 1: bsp_gather_kernel<1><<<grid, BSP_THREADS, smem, ctx->stream>>>(u, N, Ng, r, W, field, out); break;
        case 2: bsp_gather_kernel<2><<<grid, BSP_THREADS, smem, ctx->stream>>>(u, N, Ng, r, W, field, out); break;
        case 3: bsp_gather_kernel<3><<<grid, BSP_THREADS, smem, ctx->stream>>>(u, N, Ng, r, W, field, out); break;
        default: bsp_gather_kernel<5><<<grid, BSP_THREADS, smem, ctx->stream>>>(u, N, Ng, r, W, field, out); break;
        }
    }
    KDE_LAUNCHED(ctx, "bsp_gather_kernel");
    return KDE_OK;
}

// ---------------------------------------------------------------------------
// Standard-PIC step pieces for pic_step (shape_order > 0): deposit straight
// into the step's int64 accumulators, and gather + leap-frog push in place
// (no reordering: the shapes need no sorted order).
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(BSP_THREADS)
    bsp_gather_push_kernel(uint32_t *u, float *v, int64_t N, int Ng, float r, int W, const float *__restrict__ field,
                           float kick_qm_dt, float dt_scale)
{
    extern __shared__ float sf[];
    for (int g = threadIdx.x; g < Ng; g += BSP_THREADS) sf[g] = field[g];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * BSP_THREADS + threadIdx.x; i < N; i += (int64_t)gridDim.x * BSP_THREADS) {
        const uint32_t ui = u[i];
        const uint64_t q = (uint64_t)ui * (uint64_t)Ng;
        const int cell = (int)(q >> 32);
        const float frac = (float)(uint32_t)q * (1.0f / 4294967296.0f);
        float e = 0.f;
        for (int k = -W; k <= W; ++k) {
            const float b = bsp_eval<P>(((float)k - frac) * r);
            int g = (cell + k) % Ng;
            g = g < 0 ? g + Ng : g;
            e = fmaf(b, sf[g], e);
        }
        const float vn = v[i] + kick_qm_dt * (e * r);
        v[i] = vn;
        // u += rint(v dt / L 2^32) modulo 2^32 (periodic wrap for free)
        float d = vn * dt_scale;
        if (!(fabsf(d) < 2147483520.0f)) d = fmodf(d, 4294967296.0f);
        u[i] = ui + (uint32_t)(long long)__float2ll_rn(d);
    }
}

kde_status kde_bspline_deposit_acc(kde_ctx *ctx, const uint32_t *u, int64_t N, int order, double h, int Ng, double L,
                                   long long *acc, double *bound_out)
{
    const double dx = L / Ng;
    const float r = (float)(dx / h);
    const int W = bsp_window(order, h, dx);
    const double wcoef = (L / (double)N) / h;
    const double bound = (double)N * wcoef * bsp_peak(order) * 1.0000001;
    const double scale = kde_acc_scale(bound);
    *bound_out = bound;
    KDE_CUDA(ctx, cudaMemsetAsync(acc, 0, (size_t)Ng * 8, ctx->stream), "bspline acc memset");
    const int grid = bsp_grid(ctx, N);
    const size_t smem = (size_t)Ng * 8;
    {
        KdeProfScope _ps(ctx, PROF_DEPOSIT);
        switch (order) {
        case 1: bsp_deposit_kernel<1><<<grid, BSP_THREADS, smem, ctx->stream>>>(u, N, Ng, r, W, (float)wcoef, scale, acc); break;
        case 2: bsp_deposit_kernel<2><<<grid, BSP_THREADS, smem, ctx->stream>>>(u, N, Ng, r, W, (float)wcoef, scale, acc); break;
        case 3: bsp_deposit_kernel<3><<<grid, BSP_THREADS, smem, ctx->stream>>>(u, N, Ng, r, W, (float)wcoef, scale, acc); break;
        default: bsp_deposit_kernel<5><<<grid, BSP_THREADS, smem, ctx->stream>>>(u, N, Ng, r, W, (float)wcoef, scale, acc); break;
        }
    }
    KDE_LAUNCHED(ctx, "bsp_deposit_kernel");
    return KDE_OK;
}

kde_status kde_bspline_gather_push(kde_ctx *ctx, uint32_t *u, float *v, int64_t N, int order, double h, int Ng,
                                   double L, const float *E, double kick_qm_dt, double dt_scale)
{
    const double dx = L / Ng;
    const float r = (float)(dx / h);
    const int W = bsp_window(order, h, dx);
    const int grid = bsp_grid(ctx, N);
    const size_t smem = (size_t)Ng * 4;
    const float kq = (float)kick_qm_dt, ds = (float)dt_scale;
    {
        KdeProfScope _ps(ctx, PROF_GATHER);
        switch (order) {
        case 1: bsp_gather_push_kernel<1><<<grid, BSP_THREADS, smem, ctx->stream>>>(u, v, N, Ng, r, W, E, kq, ds); break;
        case 2: bsp_gather_push_kernel<2><<<grid, BSP_THREADS, smem, ctx->stream>>>(u, v, N, Ng, r, W, E, kq, ds); break;
        case 3: bsp_gather_push_kernel<3><<<grid, BSP_THREADS, smem, ctx->stream>>>(u, v, N, Ng, r, W, E, kq, ds); break;
        default: bsp_gather_push_kernel<5><<<grid, BSP_THREADS, smem, ctx->stream>>>(u, v, N, Ng, r, W, E, kq, ds); break;
        }
    }
    KDE_LAUNCHED(ctx, "bsp_gather_push_kernel");
    return KDE_OK;
}
