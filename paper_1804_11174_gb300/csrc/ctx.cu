// ctx.cu -- context, workspace, cached grid tables, position packing, damping
// rate and the throughput probes of the KDE-PIC library.
#include <cstdarg>
#include <cstring>

#include "common.cuh"

kde_status kde_fail(kde_ctx *ctx, kde_status code, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

kde_status kde_cuda_check(kde_ctx *ctx, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return KDE_OK;
    return kde_fail(ctx, e == cudaErrorMemoryAllocation ? KDE_ENOMEM : KDE_ECUDA, "%s: %s", what,
                    cudaGetErrorString(e));
}

void *kde_ws(kde_ctx *ctx, WsSlot slot, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~(size_t)255;
    if (ctx->ws_bytes[slot] >= bytes) return ctx->ws[slot];
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(ctx->stream, &cap);
    if (cap != cudaStreamCaptureStatusNone) {
        kde_fail(ctx, KDE_ENOMEM, "workspace slot %d must grow to %zu bytes during stream capture; call "
                 "kde_reserve before capturing", (int)slot, bytes);
        return nullptr;
    }
    if (ctx->ws[slot]) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->ws[slot]);
        ctx->ws[slot] = nullptr;
        ctx->ws_bytes[slot] = 0;
    }
    // grow geometrically so that slowly increasing sizes do not reallocate often
    size_t want = bytes + bytes / 4;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        kde_fail(ctx, KDE_ENOMEM, "workspace allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
        return nullptr;
    }
    ctx->ws[slot] = p;
    ctx->ws_bytes[slot] = want;
    return p;
}

double kde_host_i0e(double x) { return kde_i0e(x); }

// ---------------------------------------------------------------------------
// cached tables
// ---------------------------------------------------------------------------
// node table: (sin(theta_g/2), cos(theta_g/2)), theta_g = 2 pi g / Ng, in FP64
template <typename T2>
__global__ void node_table_kernel(T2 *tab, int Ng)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Ng) return;
    double s, c;
    sincospi((double)g / (double)Ng, &s, &c);
    tab[g].x = s;
    tab[g].y = c;
}

const void *kde_node_table(kde_ctx *ctx, int Ng, bool f64)
{
    auto key = std::make_pair(Ng, f64 ? 1 : 0);
    auto it = ctx->node_tab.find(key);
    if (it != ctx->node_tab.end()) return it->second;
    void *p = nullptr;
    size_t bytes = (size_t)Ng * (f64 ? sizeof(double2) : sizeof(float2));
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        kde_fail(ctx, KDE_ENOMEM, "node table allocation failed");
        return nullptr;
    }
    if (f64) node_table_kernel<double2><<<(Ng + 255) / 256, 256, 0, ctx->stream>>>((double2 *)p, Ng);
    else node_table_kernel<float2><<<(Ng + 255) / 256, 256, 0, ctx->stream>>>((float2 *)p, Ng);
    if (cudaGetLastError() != cudaSuccess) {
        kde_fail(ctx, KDE_ECUDA, "node table kernel launch failed");
        return nullptr;
    }
    ctx->node_tab[key] = p;
    return p;
}

// Green's function of the periodic Poisson solve, E_j = sum_l G[(j - l) mod Ng] rho_l:
//   G[d] = (1/Ng) sum_{m=1}^{M} 2 sin(2 pi m d / Ng) / q_m,  M = floor((Ng-1)/2),
// q_m = 2 pi m / L (spectral: E_m = rho_m / (i k_m)) or (2/dx) tan(pi m / Ng)
// (the finite-difference scheme of Sec. III.A in Fourier form).  Pairing modes
// m and -m gives the sine; the mean and, for even Ng, the Nyquist mode carry no
// field.  Evaluated in FP64: first the tables sin(2 pi k / Ng), k < Ng, and 1/q_m,
// then one block per d sums the M terms with the angle index m d mod Ng carried
// exactly in integers.
__global__ void green_tables_kernel(double *sinT, double *invq, int Ng, double L, int fd)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < Ng) sinT[k] = sinpi(2.0 * (double)k / Ng);
    const int M = (Ng - 1) / 2;
    if (k >= 1 && k <= M) invq[k] = 1.0 / (fd ? (2.0 * Ng / L) * tan(KDE_PI * k / Ng) : KDE_TWO_PI * k / L);
}

#define GREEN_THREADS 128
template <typename T>
__global__ void __launch_bounds__(GREEN_THREADS) green_kernel(T *G, int Ng, const double *sinT, const double *invq)
{
    __shared__ double red[GREEN_THREADS];
    const int d = blockIdx.x, M = (Ng - 1) / 2;
    const int m0 = 1 + threadIdx.x;
    const int step = (int)(((long long)GREEN_THREADS * d) % Ng);
    int r = (int)(((long long)m0 * d) % Ng);  // m d mod Ng for this thread's m
    double acc = 0.0;
    for (int m = m0; m <= M; m += GREEN_THREADS) {
        acc += sinT[r] * invq[m];
        r += step;
        if (r >= Ng) r -= Ng;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = GREEN_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) G[d] = (T)(2.0 * red[0] / Ng);
}

const void *kde_green_table(kde_ctx *ctx, int Ng, double L, bool fd, bool f64)
{
    uint64_t lb;
    std::memcpy(&lb, &L, sizeof lb);
    auto key = std::make_tuple(Ng, lb, fd ? 1 : 0, f64 ? 1 : 0);
    auto it = ctx->green_tab.find(key);
    if (it != ctx->green_tab.end()) return it->second;
    void *p = nullptr;
    if (cudaMalloc(&p, (size_t)Ng * (f64 ? 8 : 4)) != cudaSuccess) {
        cudaGetLastError();
        kde_fail(ctx, KDE_ENOMEM, "Green's function allocation failed");
        return nullptr;
    }
    // scratch for the sine and 1/q tables (a slot of its own: no caller holds it)
    double *sinT = (double *)kde_ws(ctx, WS_GREEN, (size_t)2 * KDE_MAX_NG * 8);
    if (!sinT) {
        cudaFree(p);
        return nullptr;
    }
    double *invq = sinT + KDE_MAX_NG;
    green_tables_kernel<<<(Ng + 127) / 128, 128, 0, ctx->stream>>>(sinT, invq, Ng, L, fd ? 1 : 0);
    if (f64) green_kernel<double><<<Ng, GREEN_THREADS, 0, ctx->stream>>>((double *)p, Ng, sinT, invq);
    else green_kernel<float><<<Ng, GREEN_THREADS, 0, ctx->stream>>>((float *)p, Ng, sinT, invq);
    if (cudaGetLastError() != cudaSuccess) {
        kde_fail(ctx, KDE_ECUDA, "Green's function kernel launch failed");
        return nullptr;
    }
    ctx->green_tab[key] = p;
    return p;
}

// the width-normalisation table of kde_norm_tab: q(t) = I0e(e^t) sqrt(1 + 2 pi e^t) and
// h dq/dt (central difference of step 1e-4 in t, error ~1e-9) at t = T0 + i h, in FP64
__global__ void norm_tab_kernel(float2 *tab)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= KDE_NTAB_N) return;
    const double t = KDE_NTAB_T0 + i / KDE_NTAB_INVH, d = 1e-4;
    auto q = [](double tt) {
        const double k = exp(tt);
        return kde_i0e(k) * sqrt(1.0 + KDE_TWO_PI * k);
    };
    tab[i] = make_float2((float)q(t), (float)((q(t + d) - q(t - d)) / (2.0 * d) / KDE_NTAB_INVH));
}

// ---------------------------------------------------------------------------
// C ABI: context
// ---------------------------------------------------------------------------
extern "C" kde_status kde_create(kde_ctx **out, int device, void *stream)
{
    if (!out) return KDE_EINVAL;
    *out = nullptr;
    kde_ctx *ctx = new kde_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, 4 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, 4 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->norm_tab, KDE_NTAB_N * sizeof(float2));
    if (e == cudaSuccess) {
        norm_tab_kernel<<<(KDE_NTAB_N + 255) / 256, 256, 0, ctx->stream>>>(ctx->norm_tab);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (ctx->d_status) cudaFree(ctx->d_status);
        if (ctx->norm_tab) cudaFree(ctx->norm_tab);
        delete ctx;
        return KDE_ECUDA;
    }
    *out = ctx;
    return KDE_OK;
}

extern "C" kde_status kde_destroy(kde_ctx *ctx)
{
    if (!ctx) return KDE_EINVAL;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (int i = 0; i < WS_NSLOTS; ++i)
        if (ctx->ws[i]) cudaFree(ctx->ws[i]);
    for (auto &kv : ctx->node_tab) cudaFree(kv.second);
    for (auto &kv : ctx->green_tab) cudaFree(kv.second);
    if (ctx->ad_tab) cudaFree(ctx->ad_tab);
    if (ctx->norm_tab) cudaFree(ctx->norm_tab);
    if (ctx->d_status) cudaFree(ctx->d_status);
    for (auto &p : ctx->prof) {
        cudaEventDestroy(p.second.first);
        cudaEventDestroy(p.second.second);
    }
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    delete ctx;
    return KDE_OK;
}

extern "C" kde_status kde_set_stream(kde_ctx *ctx, void *stream)
{
    if (!ctx) return KDE_EINVAL;
    ctx->stream = (cudaStream_t)stream;
    return KDE_OK;
}

extern "C" kde_status kde_set_autotune(kde_ctx *ctx, int32_t enable)
{
    if (!ctx) return KDE_EINVAL;
    ctx->autotune = enable != 0;
    return KDE_OK;
}

extern "C" kde_status kde_set_truncation(kde_ctx *ctx, double log2_cut)
{
    if (!ctx) return KDE_EINVAL;
    if (!(log2_cut == 0.0 || (log2_cut >= 16.0 && log2_cut <= 40.0)))
        return kde_fail(ctx, KDE_EINVAL, "kde_set_truncation: 0 (automatic) or a cut exponent in [16, 40]");
    ctx->cut_fixed = log2_cut;
    return KDE_OK;
}

extern "C" kde_status kde_autotune_table(const kde_ctx *ctx, int32_t cap, uint64_t *keys, int32_t *kinds,
                                         double *values, int32_t *n_out)
{
    if (!ctx || !n_out || cap < 0 || (cap > 0 && (!keys || !kinds || !values))) return KDE_EINVAL;
    int32_t n = 0;
    for (const auto &e : ctx->gat2_tuned) {
        if (n < cap) {
            keys[n] = e.first;
            kinds[n] = 0;
            values[n] = (double)e.second;
        }
        ++n;
    }
    for (const auto &e : ctx->cut_tuned) {
        if (n < cap) {
            keys[n] = e.first;
            kinds[n] = 1;
            values[n] = (double)e.second;
        }
        ++n;
    }
    *n_out = n;
    return KDE_OK;
}

extern "C" kde_status kde_autotune_set(kde_ctx *ctx, int32_t n, const uint64_t *keys, const int32_t *kinds,
                                       const double *values)
{
    if (!ctx || n < 0 || (n > 0 && (!keys || !kinds || !values))) return KDE_EINVAL;
    for (int32_t i = 0; i < n; ++i) {
        const bool shape = kinds[i] == 0 && values[i] >= 0.0 && values[i] < 3.0 && values[i] == (double)(int)values[i];
        const bool cut = kinds[i] == 1 && (values[i] == 24.0 || values[i] == 20.0 || values[i] == 18.0);
        if (!shape && !cut)
            return kde_fail(ctx, KDE_EINVAL, "kde_autotune_set: entry %d is neither a tile shape 0-2 nor a cut 24/20/18", i);
    }
    for (int32_t i = 0; i < n; ++i) {
        if (kinds[i] == 0) ctx->gat2_tuned[keys[i]] = (int)values[i];
        else ctx->cut_tuned[keys[i]] = (float)values[i];
    }
    return KDE_OK;
}

extern "C" kde_status kde_set_launch_overlap(kde_ctx *ctx, int32_t enable)
{
    if (!ctx) return KDE_EINVAL;
    ctx->overlap = enable != 0;
    return KDE_OK;
}

extern "C" kde_status kde_set_wait_limit(kde_ctx *ctx, int64_t polls)
{
    if (!ctx) return KDE_EINVAL;
    if (polls > 0xFFFFFFFFll) return kde_fail(ctx, KDE_EINVAL, "kde_set_wait_limit: at most 2^32 - 1 polls");
    ctx->wait_polls = polls < 0 ? (1u << 26) : (unsigned)polls;
    return KDE_OK;
}

extern "C" kde_status kde_autotune_entries(const kde_ctx *ctx, int32_t *n_out)
{
    if (!ctx || !n_out) return KDE_EINVAL;
    *n_out = (int32_t)ctx->gat2_tuned.size();
    return KDE_OK;
}

extern "C" const char *kde_last_error(const kde_ctx *ctx)
{
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

extern "C" kde_status kde_sync(kde_ctx *ctx)
{
    if (!ctx) return KDE_EINVAL;
    KDE_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "stream synchronize");
    unsigned int h[2] = {0, 0};
    KDE_CUDA(ctx, cudaMemcpy(h, ctx->d_status, sizeof h, cudaMemcpyDeviceToHost), "status read");
    if (h[0] != 0) {
        cudaMemset(ctx->d_status, 0, sizeof h);
        const char *what = h[0] == KDE_DEV_KAPPA_RANGE    ? "a particle width was outside (0, 1e6]"
                           : h[0] == KDE_DEV_WAIT_TIMEOUT ? "a kernel wait ran out of iterations"
                                                          : "a kernel rejected its arguments";
        return kde_fail(ctx, KDE_EDEVICE, "device status %u (detail %u): %s", h[0], h[1], what);
    }
    return KDE_OK;
}

extern "C" kde_status kde_reserve(kde_ctx *ctx, int64_t N, int32_t Ng, int32_t n_cand)
{
    if (!ctx || N < 0 || Ng < 1 || Ng > KDE_MAX_NG || n_cand < 0 || n_cand > 256)
        return kde_fail(ctx, KDE_EINVAL, "kde_reserve: bad sizes");
    cudaSetDevice(ctx->device);
    // the sizes below mirror what the kernels request (see each translation unit)
    int64_t Np = (N + 1023) / 1024 * 1024 + 1024;
    const size_t big[][2] = {
        {WS_SORT_COUNTS, (size_t)(1 << 22) * 8}, {WS_SORT_STARTS, 2048 * 4 + 64}, {WS_SORT_U, (size_t)Np * 4},
        {WS_SORT_P0, (size_t)Np * 8}, {WS_SORT_P1, (size_t)Np * 8}, {WS_SORT_P2, (size_t)Np * 8},
        {WS_SORT_P3, (size_t)Np * 4}, {WS_SORT_P1B, (size_t)Np * 8}, {WS_SORT_P2B, (size_t)Np * 8},
        {WS_SORT_P3B, (size_t)Np * 4}, {WS_SORT_PERM, (size_t)Np * 4}, {WS_NORM, (size_t)Np * 8},
        {WS_ACC, (size_t)(n_cand > 0 ? n_cand : 1) * 8192 * 8 + 64}, {WS_GRID0, KDE_MAX_NG * 8},
        {WS_GRID1, KDE_MAX_NG * 8}, {WS_GREEN, 2 * KDE_MAX_NG * 8}, {WS_WMAX, 64}, {WS_PIC_E, (size_t)Np * 4}, {WS_PIC_LOO, (size_t)Np * 4},
        {WS_PIC_KS, 64}};
    for (auto &b : big)
        if (!kde_ws(ctx, (WsSlot)b[0], b[1])) return KDE_ENOMEM;
    if (!kde_node_table(ctx, Ng, false) || !kde_node_table(ctx, Ng, true)) return KDE_ENOMEM;
    if (N > 0) KDE_TRY(kde_deposit_reserve(ctx, N, Ng));
    return KDE_OK;
}

// ---------------------------------------------------------------------------
// position packing
// ---------------------------------------------------------------------------
// u = floor(frac(x / L) * 2^32): an IEEE division (not a multiplication by a
// rounded 1/L), so that the code is the correctly rounded quotient's.  frac
// wraps negative positions and positions >= L; a fraction that rounds up to 1
// (tiny negative x) clamps to the last code.
__global__ void pack_kernel(const double *x, int64_t N, double L, uint32_t *u)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double t = __ddiv_rn(x[i], L);
    t -= floor(t);
    double q = floor(t * 4294967296.0);
    if (q > 4294967295.0) q = 4294967295.0;
    if (!(q >= 0.0)) q = 0.0;  // NaN positions map to 0
    u[i] = (uint32_t)q;
}

extern "C" kde_status kde_pack_positions(kde_ctx *ctx, const double *x, int64_t N, double L, uint32_t *u_out)
{
    if (!ctx) return KDE_EINVAL;
    if (N < 0 || !(L > 0) || (N > 0 && (!x || !u_out)))
        return kde_fail(ctx, KDE_EINVAL, "kde_pack_positions: need N >= 0, L > 0 and non-null arrays");
    if (N == 0) return KDE_OK;
    cudaSetDevice(ctx->device);
    pack_kernel<<<(unsigned)((N + 255) / 256), 256, 0, ctx->stream>>>(x, N, L, u_out);
    KDE_LAUNCHED(ctx, "pack_kernel");
    return KDE_OK;
}

// ---------------------------------------------------------------------------
// damping rate (host; Sec. III.B)
// ---------------------------------------------------------------------------
extern "C" kde_status kde_damping_rate(const double *W, int64_t n, double dt, double *gamma_out)
{
    if (!W || !gamma_out || n < 3 || !(dt > 0)) return KDE_EINVAL;
    int64_t idx[2];
    int found = 0;
    for (int64_t k = 1; k + 1 < n && found < 2; ++k)
        if (W[k] > W[k - 1] && W[k] > W[k + 1]) idx[found++] = k;
    if (found < 2) return KDE_EINVAL;
    *gamma_out = 0.5 * (std::log(W[idx[1]]) - std::log(W[idx[0]])) / ((double)(idx[1] - idx[0]) * dt);
    return KDE_OK;
}

// ---------------------------------------------------------------------------
// throughput probes: independent chains, 8 per thread, so that the pipe and not
// the dependency latency limits the rate
// ---------------------------------------------------------------------------
__global__ void probe_exp2_kernel(int64_t iters, float seed, float *sink)
{
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = -1e-3f * (threadIdx.x + k) * seed;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = kde_ex2(a[k]) - 1.0001f;
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == 12345.f) sink[0] = s;
}

__global__ void probe_fma_kernel(int64_t iters, float seed, float *sink)
{
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 1e-3f * (threadIdx.x + k) * seed;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], 0.999f, 1e-7f);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == 12345.f) sink[0] = s;
}

static kde_status run_probe(kde_ctx *ctx, int which, int64_t iters, double *ms_out, int64_t *ops_out)
{
    if (!ctx || iters < 1 || !ms_out) return kde_fail(ctx, KDE_EINVAL, "probe: bad arguments");
    cudaSetDevice(ctx->device);
    float *sink = (float *)kde_ws(ctx, WS_WMAX, 64);
    if (!sink) return KDE_ENOMEM;
    int blocks = ctx->sm_count * 4, threads = 512;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    // warm-up
    if (which == 0) probe_exp2_kernel<<<blocks, threads, 0, ctx->stream>>>(iters / 8 + 1, 1.0f, sink);
    else probe_fma_kernel<<<blocks, threads, 0, ctx->stream>>>(iters / 8 + 1, 1.0f, sink);
    cudaEventRecord(a, ctx->stream);
    if (which == 0) probe_exp2_kernel<<<blocks, threads, 0, ctx->stream>>>(iters, 1.0f, sink);
    else probe_fma_kernel<<<blocks, threads, 0, ctx->stream>>>(iters, 1.0f, sink);
    cudaEventRecord(b, ctx->stream);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    KDE_CUDA(ctx, e, "probe");
    *ms_out = ms;
    if (ops_out) *ops_out = (int64_t)blocks * threads * 8 * iters;
    return KDE_OK;
}

extern "C" kde_status kde_probe_exp2(kde_ctx *ctx, int64_t iters, double *ms_out, int64_t *ops_out)
{
    return run_probe(ctx, 0, iters, ms_out, ops_out);
}

extern "C" kde_status kde_probe_fma(kde_ctx *ctx, int64_t iters, double *ms_out, int64_t *ops_out)
{
    return run_probe(ctx, 1, iters, ms_out, ops_out);
}

// ---------------------------------------------------------------------------
// profiling hook
// ---------------------------------------------------------------------------
cudaEvent_t kde_prof_event(kde_ctx *ctx)
{
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

extern "C" kde_status kde_profile_enable(kde_ctx *ctx, int on)
{
    if (!ctx) return KDE_EINVAL;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto &p : ctx->prof) {
        ctx->ev_pool.push_back(p.second.first);
        ctx->ev_pool.push_back(p.second.second);
    }
    ctx->prof.clear();
    ctx->launches = 0;
    ctx->prof_on = on != 0;
    return KDE_OK;
}

extern "C" kde_status kde_profile_read(kde_ctx *ctx, int kernel, double *total_ms, int64_t *launches)
{
    if (!ctx || kernel < -1 || kernel >= PROF_NIDS) return KDE_EINVAL;
    cudaSetDevice(ctx->device);
    KDE_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "profile synchronize");
    if (kernel == -1) {  // all kernel launches of the library since kde_profile_enable
        if (launches) *launches = ctx->launches;
        if (total_ms) *total_ms = 0.0;
        return KDE_OK;
    }
    double ms = 0.0;
    int64_t n = 0;
    for (auto &p : ctx->prof)
        if (p.first == kernel) {
            float t = 0.f;
            cudaEventElapsedTime(&t, p.second.first, p.second.second);
            ms += t;
            ++n;
        }
    if (total_ms) *total_ms = ms;
    if (launches) *launches = n;
    return KDE_OK;
}
