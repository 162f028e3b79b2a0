// gather.cu -- field interpolation through the deposit's kernels, fused with
// the leap-frog push of the PIC cycle (Sec. III.A).
//
//   E_i = (2 pi / Ng) norm(kappa_i) sum_g E_g exp(-2 kappa_i sin^2((theta_g - theta_i)/2))
//
// Layout: the whole grid (half-angle sine, cosine, field) sits in shared
// memory.  Threads own particles (cell-sorted, so a warp's particles share a
// few cells); each warp sweeps one node window covering all of its lanes'
// truncated supports, so every node read is a shared-memory broadcast.  The
// push, the write-back of the particle state and (block 0) the field energy
// ride in the same kernel.
#include "common.cuh"

#define GAT_THREADS 256

struct __align__(16) GNodeD {
    double x, y, z, w;
};
template <typename T> struct GNode;
template <> struct GNode<float> { typedef float4 t; };
template <> struct GNode<double> { typedef GNodeD t; };

template <typename T> struct V2g;
template <> struct V2g<float> { typedef float2 t; };
template <> struct V2g<double> { typedef double2 t; };

template <typename T> struct GatherArgs {
    const uint32_t *u;
    const T *kappa;
    T kappa_u;
    const T *norm;
    T norm_u;
    int64_t N;
    const T *field;
    int Ng;
    const typename V2g<T>::t *nodes;
    T coef;  // 2 pi / Ng
    T *out;
    const uint32_t *perm;
    // push (active when u_out != nullptr)
    const T *v_in;
    uint32_t *u_out;
    T *v_out;
    T *kappa_out;
    const T *norm_in;
    T *norm_out;
    const uint32_t *id_in;
    uint32_t *id_out;
    T kick_qm_dt;
    T dt_scale;
    double *energy;
    const double *kstar_in;
    double *kstar_out;
    double dx;
    unsigned int *status;
    const float2 *ntab;  // FP32 norm table (kde_norm_tab): per-particle widths without norms
    // push only: count table of the next step's cell sort, or null (counts of the new
    // positions are added with one atomic per warp and distinct cell)
    unsigned int *counts;
    int cnt_nblk, cnt_shift;
    float xcut = (float)KDE_XCUT;  // FP32 packed gather: truncation cut exponent
};

__device__ __forceinline__ int window_nodes_g(float kappa, int Ng, float xcut)
{
    float s2 = xcut * (float)(KDE_LN2 / 2.0) / kappa;
    if (s2 >= 1.0f) return Ng;
    float r = 2.0f * asinf(sqrtf(s2));
    int w = (int)ceilf(r * (float)Ng * (float)(1.0 / KDE_TWO_PI)) + 1;
    return w >= Ng ? Ng : w;
}

__device__ __forceinline__ uint32_t advance_position(uint32_t u, float d)
{
    // d = displacement in units of 2^-32 L
    if (fabsf(d) < 2147483520.0f) return u + (uint32_t)__float2int_rn(d);
    d = fmodf(d, 4294967296.0f);
    return u + (uint32_t)(long long)__float2ll_rn(d);
}
__device__ __forceinline__ uint32_t advance_position(uint32_t u, double d)
{
    d = fmod(d, 4294967296.0);
    return u + (uint32_t)(long long)__double2ll_rn(d);
}

template <typename T>
__global__ void __launch_bounds__(GAT_THREADS) gather_kernel(GatherArgs<T> A)
{
    extern __shared__ __align__(16) unsigned char sm[];
    typename GNode<T>::t *node = (typename GNode<T>::t *)sm;
    const int Ng = A.Ng;
    for (int g = threadIdx.x; g < Ng; g += GAT_THREADS) {
        typename V2g<T>::t sc = A.nodes[g];
        typename GNode<T>::t q;
        q.x = sc.x;
        q.y = sc.y;
        q.z = A.field[g];
        q.w = 0;
        node[g] = q;
    }
    if (blockIdx.x == 0 && A.energy) {
        __shared__ double red[GAT_THREADS];
        double s = 0.0;
        for (int g = threadIdx.x; g < Ng; g += GAT_THREADS) s += (double)A.field[g] * (double)A.field[g];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int o = GAT_THREADS / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            A.energy[0] = 0.5 * red[0] * A.dx;
            if (A.kstar_out) A.kstar_out[0] = A.kstar_in ? A.kstar_in[0] : (double)A.kappa_u;
        }
    }
    __syncthreads();

    const int64_t j = (int64_t)blockIdx.x * GAT_THREADS + threadIdx.x;
    const bool valid = j < A.N;
    uint32_t uu = valid ? A.u[j] : 0u;
    T k = A.kappa ? (valid ? A.kappa[j] : (T)1) : A.kappa_u;
    if (valid && !(k > (T)0 && k <= (T)KDE_KAPPA_MAX)) {
        kde_flag(A.status, KDE_DEV_KAPPA_RANGE, (unsigned)j);
        k = (T)KDE_KAPPA_MAX;
    }
    T nm = A.norm ? (valid ? A.norm[j] : (T)0) : (A.kappa ? (T)kde_norm((double)k) : A.norm_u);
    T sh, ch;
    kde_half_sincos(uu, sh, ch);
    T beta = sqrt((T)(2.0 * KDE_LOG2E) * k);
    const T bs = beta * sh, bc = beta * ch;
    const int cell = kde_cell(uu, Ng);
    const int W = window_nodes_g((float)k, Ng, (float)KdeCut<T>::x);
    // warp-uniform window [lo, hi] covering every valid lane's support
    int lo = valid ? cell - W : 0x3fffffff, hi = valid ? cell + W : -0x3fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    int len = hi - lo + 1;
    if (len >= Ng) {
        lo = 0;
        len = Ng;
    }
    if (len <= 0) return;  // whole warp past the end
    int g = lo % Ng;
    if (g < 0) g += Ng;
    T acc0 = 0, acc1 = 0;
    int t = 0;
    for (; t + 1 < len; t += 2) {
        typename GNode<T>::t q0 = node[g];
        int g1 = g + 1 == Ng ? 0 : g + 1;
        typename GNode<T>::t q1 = node[g1];
        g = g1 + 1 == Ng ? 0 : g1 + 1;
        T s0 = q0.x * bc - q0.y * bs;
        T s1 = q1.x * bc - q1.y * bs;
        acc0 += kde_ex2(-s0 * s0) * q0.z;
        acc1 += kde_ex2(-s1 * s1) * q1.z;
    }
    if (t < len) {
        typename GNode<T>::t q0 = node[g];
        T s0 = q0.x * bc - q0.y * bs;
        acc0 += kde_ex2(-s0 * s0) * q0.z;
    }
    if (!valid) return;
    const T Ei = (acc0 + acc1) * nm * A.coef;
    if (A.u_out) {
        T v = A.v_in[j] + A.kick_qm_dt * Ei;
        A.v_out[j] = v;
        A.u_out[j] = advance_position(uu, v * A.dt_scale);
        if (A.kappa_out) A.kappa_out[j] = k;
        if (A.norm_out) A.norm_out[j] = A.norm_in[j];
        if (A.id_out) A.id_out[j] = A.id_in[j];
    } else {
        A.out[A.perm ? A.perm[j] : j] = Ei;
    }
}

// ---------------------------------------------------------------------------
// FP32 gather with packed pair arithmetic: each lane carries GAT2_NP = 4
// particles (a warp covers 128 consecutive sorted particles) as two f32x2
// pairs, and every node record is kept pre-duplicated in shared memory, so one
// 128-bit and one 64-bit broadcast load feed four particles' multiply-adds.  The
// node loop runs as two contiguous segments (before and after the wrap point), so
// it carries no per-node index arithmetic.  The form of the kernel value is chosen
// per block by its largest width, as in the packed deposit:
//  * half-angle: nodes (sin, sin, -cos, -cos) of half the node angle, particles
//    (beta sin, beta cos) of half theirs, 2^-(S_g beta c_j - C_g beta s_j)^2;
//  * cosine (largest width <= KDE_COSFORM_KMAX): nodes (sin, sin, cos, cos) of the
//    full angle, particles (K cos, K sin), 2^(K cos(x_j - x_g)), and 2^-K folded into
//    the particle's norm; three multiply-adds per pair instead of four.
// ---------------------------------------------------------------------------
// Tile shapes (template parameters of gather2_kernel, chosen per call by the variant
// table below): NP particles a lane (even), node-loop unrolling UD for windows of
// GAT2_DEEP_LEN nodes or more and US below, and a launch bound of MINB resident
// blocks per SM.  Variants with the same NP compute the same sums in the same order
// (NP sets each warp's node window), so their results are bitwise identical and only
// the speed differs.
#define GAT2_WARPS 4
#define GAT2_DEEP_LEN 128

// the node loop of the packed gather over the window's two contiguous segments
// [g0, e1) and [0, e2): NPP particle pairs a lane, U nodes unrolled
template <int U, bool COS, int NPP>
__device__ __forceinline__ void gat2_nodes(const float4 *SC, const float2 *FF, int g0, int e1, int e2,
                                           const kde_f2 (&psP)[NPP], const kde_f2 (&pcP)[NPP], kde_f2 (&acc)[NPP])
{
    auto node = [&](int g) {
        const float4 r4 = SC[g];
        const float2 f = FF[g];
        const kde_f2 S2 = kde_pk(r4.x, r4.y), C2 = kde_pk(r4.z, r4.w), F2 = kde_pk(f.x, f.y);
#pragma unroll
        for (int q = 0; q < NPP; ++q) {
            const kde_f2 ev = kde_fma2(S2, psP[q], kde_mul2(C2, pcP[q]));
            if (COS) acc[q] = kde_fma2(kde_ex22(ev), F2, acc[q]);  // 2^(K cos(x_j - x_g))
            else acc[q] = kde_fma2(kde_ex2neg2(kde_mul2(ev, ev)), F2, acc[q]);  // 2^-(beta sin((x_j - x_g)/2))^2
        }
    };
#pragma unroll U
    for (int g = g0; g < e1; ++g) node(g);
#pragma unroll U
    for (int g = 0; g < e2; ++g) node(g);
}

template <int NP, int UD, int US, int MINB>
__global__ void __launch_bounds__(GAT2_WARPS * 32, MINB) gather2_kernel(GatherArgs<float> A)
{
    constexpr int GAT2_NP = NP, GAT2_ITEM = 32 * NP;
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ float kred[GAT2_WARPS];
    const int Ng = A.Ng;
    float4 *SC = (float4 *)sm;         // node angle records
    float2 *FF = (float2 *)(SC + Ng);  // (E, E)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = ((int64_t)blockIdx.x * GAT2_WARPS + warp) * GAT2_ITEM;
    // held across the node loop: positions and norms; widths until the particle terms
    // are formed; the push's other inputs are loaded after the loop (registers are the
    // limit with eight particles a lane, and other warps cover the load latency)
    float nm[GAT2_NP], kap[GAT2_NP];
    uint32_t uu[GAT2_NP];
    int lo = 0x3fffffff, hi = -0x3fffffff;  // the warp's first and last cell, then its window
    float kmax = 0.f, kmin = (float)KDE_KAPPA_MAX;
#pragma unroll
    for (int h = 0; h < GAT2_NP; ++h) {
        const int64_t j = base + h * 32 + lane;
        const bool valid = j < A.N;
        uu[h] = valid ? A.u[j] : 0u;
        float k = A.kappa ? (valid ? A.kappa[j] : 1.0f) : A.kappa_u;
        if (valid && !(k > 0.f && k <= (float)KDE_KAPPA_MAX)) {
            kde_flag(A.status, KDE_DEV_KAPPA_RANGE, (unsigned)j);
            k = (float)KDE_KAPPA_MAX;
        }
        kap[h] = k;
        nm[h] = A.norm ? (valid ? A.norm[j] : 0.f) : (A.kappa ? kde_norm_tab(A.ntab, k) : A.norm_u);
        if (valid) {
            kmax = fmaxf(kmax, k);
            kmin = fminf(kmin, k);
            const int cell = kde_cell(uu[h], Ng);
            lo = min(lo, cell);
            hi = max(hi, cell);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        kmax = fmaxf(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        kmin = fminf(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
    }
    // one window for the warp: the widest kernel's reach around its cell range (it holds
    // every particle's own window, since the widest kernel has the smallest kappa)
    if (lo <= hi) {
        const int W = window_nodes_g(kmin, Ng, A.xcut);
        lo -= W;
        hi += W;
    }
    if (lane == 0) kred[warp] = kmax;
    __syncthreads();
#pragma unroll
    for (int w = 0; w < GAT2_WARPS; ++w) kmax = fmaxf(kmax, kred[w]);
    const bool cosf = kmax <= KDE_COSFORM_KMAX;
    for (int g = threadIdx.x; g < Ng; g += GAT2_WARPS * 32) {
        const float2 sc = A.nodes[g];
        if (cosf) {
            const float sf = 2.f * sc.x * sc.y, cf = (sc.y - sc.x) * (sc.y + sc.x);
            SC[g] = make_float4(sf, sf, cf, cf);
        } else {
            SC[g] = make_float4(sc.x, sc.x, -sc.y, -sc.y);
        }
    }
    // the field is the previous kernel's output; so far only the sorted particles (two or
    // more kernels back) and the node table have been read
    kde_pdl_wait();
    kde_pdl_trigger();
    for (int g = threadIdx.x; g < Ng; g += GAT2_WARPS * 32) {
        const float f = A.field[g];
        FF[g] = make_float2(f, f);
    }
    if (blockIdx.x == 0 && A.energy) {
        __shared__ double red[GAT2_WARPS * 32];
        double sum = 0.0;
        for (int g = threadIdx.x; g < Ng; g += GAT2_WARPS * 32) sum += (double)A.field[g] * (double)A.field[g];
        red[threadIdx.x] = sum;
        __syncthreads();
        for (int o = GAT2_WARPS * 16; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            A.energy[0] = 0.5 * red[0] * A.dx;
            if (A.kstar_out) A.kstar_out[0] = A.kstar_in ? A.kstar_in[0] : (double)A.kappa_u;
        }
    }
    __syncthreads();

    int len = hi - lo + 1;
    if (len >= Ng) {
        lo = 0;
        len = Ng;
    }
    if (len <= 0) return;  // whole warp past the end
    // (ps, pc) pair with the node's (sin, sin) and (c, c) columns: half-angle (beta cos,
    // beta sin) of half the particle angle, cosine form (K sin, K cos) of the full one
    float ps[GAT2_NP], pc[GAT2_NP];
#pragma unroll
    for (int h = 0; h < GAT2_NP; ++h) {
        float sh, ch;
        kde_half_sincos(uu[h], sh, ch);
        if (cosf) {
            const float K = (float)KDE_LOG2E * kap[h];
            ps[h] = K * (2.f * sh * ch);
            pc[h] = K * ((ch - sh) * (ch + sh));
            nm[h] *= kde_ex2(-K);
        } else {
            const float beta = sqrtf((float)(2.0 * KDE_LOG2E) * kap[h]);
            ps[h] = beta * ch;
            pc[h] = beta * sh;
        }
    }
    int g0 = lo % Ng;
    if (g0 < 0) g0 += Ng;
    constexpr int NPP = GAT2_NP / 2;  // packed particle pairs a lane
    kde_f2 psP[NPP], pcP[NPP], acc[NPP];
#pragma unroll
    for (int q = 0; q < NPP; ++q) {
        psP[q] = kde_pk(ps[2 * q], ps[2 * q + 1]);
        pcP[q] = kde_pk(pc[2 * q], pc[2 * q + 1]);
        acc[q] = kde_pk(0.f, 0.f);
    }
    const int e1 = g0 + len < Ng ? g0 + len : Ng;  // first segment [g0, e1), then [0, len - (e1 - g0))
    const int e2 = len - (e1 - g0);
    // long windows take the deeper unrolling (more exp2 in flight), short ones the
    // shallower (less remainder work)
    const bool deep = len >= GAT2_DEEP_LEN;
    if (cosf) {
        if (deep) gat2_nodes<UD, true, NPP>(SC, FF, g0, e1, e2, psP, pcP, acc);
        else gat2_nodes<US, true, NPP>(SC, FF, g0, e1, e2, psP, pcP, acc);
    } else {
        if (deep) gat2_nodes<UD, false, NPP>(SC, FF, g0, e1, e2, psP, pcP, acc);
        else gat2_nodes<US, false, NPP>(SC, FF, g0, e1, e2, psP, pcP, acc);
    }
    float ea[GAT2_NP];
#pragma unroll
    for (int q = 0; q < NPP; ++q) kde_upk(acc[q], ea[2 * q], ea[2 * q + 1]);
    if (A.u_out) {
        // the push's inputs of four particles at a time first (one load latency per group;
        // the stores below alias nothing the loads read, but the compiler cannot know
        // that), then the stores
        constexpr int HB = GAT2_NP % 4 == 0 ? 4 : (GAT2_NP % 3 == 0 ? 3 : 2);
#pragma unroll
        for (int h0 = 0; h0 < GAT2_NP; h0 += HB) {
        float vin[HB], kin[HB], nin[HB];
        uint32_t idin[HB];
#pragma unroll
        for (int hh = 0; hh < HB; ++hh) {
            const int64_t j = base + (h0 + hh) * 32 + lane;
            const bool ok = j < A.N;
            vin[hh] = ok ? A.v_in[j] : 0.f;
            kin[hh] = (ok && A.kappa_out) ? (A.kappa ? A.kappa[j] : A.kappa_u) : 0.f;
            nin[hh] = (ok && A.norm_out) ? A.norm_in[j] : 0.f;
            idin[hh] = (ok && A.id_out) ? A.id_in[j] : 0u;
        }
#pragma unroll
        for (int hh = 0; hh < HB; ++hh) {
            const int h = h0 + hh;
            const int64_t j = base + h * 32 + lane;
            int key = -1;
            if (j < A.N) {
                const float v = vin[hh] + A.kick_qm_dt * (ea[h] * nm[h] * A.coef);
                A.v_out[j] = v;
                const uint32_t nu = advance_position(uu[h], v * A.dt_scale);
                A.u_out[j] = nu;
                if (A.kappa_out) {
                    const float k = kin[hh];
                    A.kappa_out[j] = (k > 0.f && k <= (float)KDE_KAPPA_MAX) ? k : (float)KDE_KAPPA_MAX;
                }
                if (A.norm_out) A.norm_out[j] = nin[hh];
                if (A.id_out) A.id_out[j] = idin[hh];
                key = kde_cell(nu, Ng);
            }
            if (A.counts) {  // warp-uniform; the 32 particles of a round share one sort tile
                const unsigned int peers = __match_any_sync(0xffffffffu, key);
                if (key >= 0 && lane == __ffs(peers) - 1)
                    atomicAdd(&A.counts[(size_t)key * A.cnt_nblk + (size_t)(j >> A.cnt_shift)],
                              (unsigned int)__popc(peers));
            }
        }
        }
    } else {
#pragma unroll
        for (int h = 0; h < GAT2_NP; ++h) {
            const int64_t j = base + h * 32 + lane;
            if (j < A.N) A.out[A.perm ? A.perm[j] : j] = ea[h] * nm[h] * A.coef;
        }
    }
}

// the tile-shape variants of the packed gather: (particles a lane, deep and short
// unrolling, launch bound)
#define GAT2_NVARIANTS 3

template <int NP, int UD, int US, int MINB>
static kde_status gat2_launch(kde_ctx *ctx, const GatherArgs<float> &A)
{
    auto kern = gather2_kernel<NP, UD, US, MINB>;
    static bool attr = false;
    if (!attr) {
        KDE_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           KDE_MAX_NG * (int)(sizeof(float4) + sizeof(float2))),
                 "gather2 attribute");
        attr = true;
    }
    const size_t smem = (size_t)A.Ng * (sizeof(float4) + sizeof(float2));
    unsigned grid = (unsigned)((A.N + GAT2_WARPS * 32 * NP - 1) / (GAT2_WARPS * 32 * NP));
    if (grid == 0) grid = 1;
    // with the push (the PIC step) the kernel before is the field kernel, which writes
    // none of the sorted particle arrays the prologue reads before its wait; a plain
    // gather may follow the sort that wrote them, so it starts after it as usual
    KDE_CUDA(ctx, kde_launch(ctx, A.u_out != nullptr, kern, dim3(grid), dim3(GAT2_WARPS * 32), smem, A),
             "gather2_kernel");
    KDE_LAUNCHED(ctx, "gather2_kernel");
    return KDE_OK;
}

static kde_status gat2_variant(kde_ctx *ctx, const GatherArgs<float> &A, int v)
{
    // all with four particles a lane: the warps' particle sets, and so their node windows
    // and kernel forms, are the same in every variant.  Launch bounds of 6, 7 and 8 blocks
    // an SM; the default 7 (71 registers) puts a Landau-size run (2048 blocks) in two
    // nearly full waves and measured best or within 1% of best from whole-grid to
    // five-node windows.  (Eight particles a lane, which makes a Landau-size run one
    // wave, measured 10% slower: the 64-register bound leaves the node loop less room.)
    switch (v) {
    case 1: return gat2_launch<4, 4, 4, 8>(ctx, A);
    case 2: return gat2_launch<4, 8, 4, 6>(ctx, A);
    default: return gat2_launch<4, 8, 4, 7>(ctx, A);
    }
}

static uint64_t gat2_key(const GatherArgs<float> &A)
{
    return kde_width_key(A.N, A.Ng, A.kappa != nullptr, (double)A.kappa_u);
}

// the variant for this call: the tuned one for its key; with autotuning on and no stream
// capture, a key seen for the first time is tuned on this call's own data (every variant
// runs twice, timed by events on the stream, the fastest second run wins), provided that
// repeating the call cannot change its result (no output aliases an input)
static kde_status launch_gather2(kde_ctx *ctx, GatherArgs<float> &A)
{
    const void *nodes = kde_node_table(ctx, A.Ng, false);
    if (!nodes) return KDE_ENOMEM;
    A.nodes = (const float2 *)nodes;
    A.status = ctx->d_status;
    A.ntab = ctx->norm_tab;
    const uint64_t key = gat2_key(A);
    auto it = ctx->gat2_tuned.find(key);
    int v = it != ctx->gat2_tuned.end() ? it->second : 0;
    bool tune = false;
    if (it == ctx->gat2_tuned.end() && ctx->autotune) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(ctx->stream, &cap);
        auto apart = [](const void *out, const void *in) { return !out || out != in; };
        const bool idem = !A.u_out || (apart(A.u_out, A.u) && apart(A.v_out, A.v_in) && apart(A.kappa_out, A.kappa) &&
                                       apart(A.norm_out, A.norm_in) && apart(A.norm_out, A.norm) &&
                                       apart(A.id_out, A.id_in));
        tune = cap == cudaStreamCaptureStatusNone && idem;
    }
    if (!tune) {
        KdeProfScope _ps(ctx, PROF_GATHER);
        return gat2_variant(ctx, A, v);
    }
    cudaEvent_t ev[2 * GAT2_NVARIANTS + 1];
    for (auto &e : ev) KDE_CUDA(ctx, cudaEventCreate(&e), "autotune event");
    KDE_CUDA(ctx, cudaEventRecord(ev[0], ctx->stream), "autotune event");
    // the timed runs add no sort counts (they repeat the gather); the chosen shape runs
    // once more below with the caller's arguments
    GatherArgs<float> T = A;
    T.counts = nullptr;
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < GAT2_NVARIANTS; ++k) {
            KDE_TRY(gat2_variant(ctx, T, k));
            KDE_CUDA(ctx, cudaEventRecord(ev[1 + r * GAT2_NVARIANTS + k], ctx->stream), "autotune event");
        }
    KDE_CUDA(ctx, cudaEventSynchronize(ev[2 * GAT2_NVARIANTS]), "autotune wait");
    float best = 3.0e38f;
    for (int k = 0; k < GAT2_NVARIANTS; ++k) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[GAT2_NVARIANTS + k], ev[GAT2_NVARIANTS + k + 1]);
        if (ms < best) {
            best = ms;
            v = k;
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    ctx->gat2_tuned[key] = v;
    if (A.counts) {
        KdeProfScope _ps(ctx, PROF_GATHER);
        return gat2_variant(ctx, A, v);
    }
    return KDE_OK;
}

template <typename T>
static kde_status launch_gather(kde_ctx *ctx, GatherArgs<T> &A)
{
    const void *nodes = kde_node_table(ctx, A.Ng, sizeof(T) == 8);
    if (!nodes) return KDE_ENOMEM;
    A.nodes = (const typename V2g<T>::t *)nodes;
    A.status = ctx->d_status;
    size_t smem = (size_t)A.Ng * sizeof(typename GNode<T>::t);
    static bool attr[2] = {false, false};
    if (!attr[sizeof(T) == 8]) {
        cudaFuncSetAttribute(gather_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             KDE_MAX_NG * (int)sizeof(typename GNode<T>::t));
        attr[sizeof(T) == 8] = true;
    }
    unsigned grid = (unsigned)((A.N + GAT_THREADS - 1) / GAT_THREADS);
    if (grid == 0) grid = 1;
    {
        KdeProfScope _ps(ctx, PROF_GATHER);
    gather_kernel<T><<<grid, GAT_THREADS, smem, ctx->stream>>>(A);
    }
    KDE_LAUNCHED(ctx, "gather_kernel");
    return KDE_OK;
}

template <typename T>
kde_status kde_gather_sorted(kde_ctx *ctx, const uint32_t *u, const T *kappa, T kappa_u, const T *norm, T norm_u,
                             int64_t N, const T *field, int Ng, double coef, T *out, const uint32_t *perm,
                             const PushArgs *push, float xcut)
{
    GatherArgs<T> A{};
    A.u = u;
    A.kappa = kappa;
    A.kappa_u = kappa_u;
    A.norm = norm;
    A.norm_u = norm_u;
    A.N = N;
    A.field = field;
    A.Ng = Ng;
    A.coef = (T)coef;
    A.out = out;
    A.perm = perm;
    A.xcut = xcut > 0.f ? xcut : (push && push->xcut > 0.f ? push->xcut : kde_fp32_cut(ctx));
    if (push) {
        A.v_in = (const T *)push->v_in;
        A.u_out = push->u_out;
        A.v_out = (T *)push->v_out;
        A.kappa_out = (T *)push->kappa_out;
        A.norm_in = (const T *)push->norm_in;
        A.norm_out = (T *)push->norm_out;
        A.id_in = push->id_in;
        A.id_out = push->id_out;
        A.kick_qm_dt = (T)(push->kick * push->qm_dt);
        A.dt_scale = (T)push->dt_scale;
        A.energy = push->energy;
        A.kstar_in = push->kstar_in;
        A.kstar_out = push->kstar_out;
        A.dx = push->dx;
        A.counts = push->counts;
        A.cnt_nblk = push->cnt_nblk;
        A.cnt_shift = push->cnt_shift;
    }
    if constexpr (sizeof(T) == 4) return launch_gather2(ctx, A);
    else return launch_gather<T>(ctx, A);
}

template kde_status kde_gather_sorted<float>(kde_ctx *, const uint32_t *, const float *, float, const float *, float,
                                             int64_t, const float *, int, double, float *, const uint32_t *,
                                             const PushArgs *, float);
template kde_status kde_gather_sorted<double>(kde_ctx *, const uint32_t *, const double *, double, const double *,
                                              double, int64_t, const double *, int, double, double *,
                                              const uint32_t *, const PushArgs *, float);

// ---------------------------------------------------------------------------
template <typename T>
static kde_status gather_api(kde_ctx *ctx, const uint32_t *u, const T *kappa, double kappa_u, int64_t N,
                             const T *field, int Ng, double L, T *out)
{
    cudaSetDevice(ctx->device);
    uint32_t *us = (uint32_t *)kde_ws(ctx, WS_SORT_U, (size_t)N * 4);
    uint32_t *perm = (uint32_t *)kde_ws(ctx, WS_SORT_PERM, (size_t)N * 4);
    T *ks = kappa ? (T *)kde_ws(ctx, WS_SORT_P0, (size_t)N * sizeof(T)) : nullptr;
    if (!us || !perm || (kappa && !ks)) return KDE_ENOMEM;
    SortPayload pl[1];
    int npl = 0;
    if (kappa) pl[npl++] = SortPayload{kappa, ks, (int)sizeof(T)};
    KDE_TRY(kde_sort_by_bin(ctx, u, N, Ng, us, pl, npl, perm));
    double norm_u = kappa ? 0.0 : kde_norm(kappa_u);
    return kde_gather_sorted<T>(ctx, us, ks, (T)kappa_u, nullptr, (T)norm_u, N, field, Ng, KDE_TWO_PI / Ng, out, perm,
                                nullptr);
}

extern "C" kde_status kde_gather(kde_ctx *ctx, const uint32_t *u, const void *kappa, double kappa_uniform, int64_t N,
                                 const void *field, int32_t Ng, double L, void *out, uint32_t flags)
{
    if (!ctx) return KDE_EINVAL;
    if (N < 0 || Ng < 1 || Ng > KDE_MAX_NG || !(L > 0) || !field || (N > 0 && (!u || !out)))
        return kde_fail(ctx, KDE_EINVAL, "kde_gather: need N >= 0, 1 <= Ng <= %d, L > 0, non-null arrays",
                        KDE_MAX_NG);
    if (!kappa && !(kappa_uniform > 0 && kappa_uniform <= KDE_KAPPA_MAX))
        return kde_fail(ctx, KDE_EINVAL, "kde_gather: kappa_uniform must be in (0, 1e6]");
    if (N > 0xFFFFFFFFll) return kde_fail(ctx, KDE_EINVAL, "kde_gather: N must be below 2^32");
    if (flags & ~KDE_F64) return kde_fail(ctx, KDE_ENOTSUP, "kde_gather: unsupported flags 0x%x", flags);
    if (N == 0) return KDE_OK;
    if (flags & KDE_F64)
        return gather_api<double>(ctx, u, (const double *)kappa, kappa_uniform, N, (const double *)field, Ng, L,
                                  (double *)out);
    return gather_api<float>(ctx, u, (const float *)kappa, kappa_uniform, N, (const float *)field, Ng, L,
                             (float *)out);
}
