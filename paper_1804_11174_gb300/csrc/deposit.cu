// deposit.cu -- KDE deposit (Eq. kde evaluated at the grid nodes).
//
//   rho_g = sum_i w_i (2 pi / L) norm(kappa_i) exp(-2 kappa_i sin^2((theta_g - theta_i)/2))
//
// Layout: particles are counting-sorted by cell.  One CTA takes a chunk of
// DEP_CHUNK consecutive sorted particles, stages (beta sin, beta cos, w*norm)
// of each in shared memory, and finds the node range its particles' truncated
// kernels can reach (first/last cell +- the widest window).  Lanes own nodes
// (node-owner formulation): a warp sweeps 32 consecutive nodes over a slice of
// the chunk, so every particle value is a shared-memory broadcast and each
// lane accumulates in a register without atomics.  Slices are combined in a
// fixed order in shared memory.  Chunk partials are converted to int64 fixed
// point (an exact power-of-two scale below the largest possible node value)
// and added with integer atomics, so the grid sum is exact and independent of
// the order in which chunks finish: results are bitwise reproducible.
#include "common.cuh"

#define DEP_THREADS 256
#define DEP_WARPS (DEP_THREADS / 32)
#define DEP_CHUNK 1024
#define CV_MAXM 8192

template <typename T> struct V2;
template <> struct V2<float> { typedef float2 t; };
template <> struct V2<double> { typedef double2 t; };

template <typename T> struct DepRec {
    T bs, bc, wn;
};

template <typename T> struct DepSrc {
    const uint32_t *u;
    int64_t N;
    const T *kappa;      // per-particle widths, or nullptr
    T kappa_u;           // uniform width
    T kscale;            // widths are kscale * kappa[j] (CV scale mode), else 1
    const T *norm;       // per-particle norm, or nullptr (computed from the width when kappa != nullptr)
    const float *lnorm;  // log2 of per-particle norm (CV scale mode), or nullptr
    T norm_u;            // uniform norm
    const T *w;          // per-particle weights, or nullptr
    T w_u;               // uniform weight
    T coef;              // 2 pi / L (x units) or 1 (theta units)
    int Ng;
    const typename V2<T>::t *nodes;  // (sin, cos) of half node angles; nullptr: Ng is a power of two
    long long *acc;
    double bound;                    // largest possible node value
    const unsigned int *wmax_bits;   // if not null: bound = N * coef * norm_bound * w_max (float bits)
    double norm_bound;
    unsigned int *status;
    int scale_exp;  // KDE_ES_FROM_BOUND, or the exponent es of the fixed-point scale 2^es
    const float2 *ntab;  // FP32 norm table (kde_norm_tab) for per-particle widths without norms, or nullptr
    float xcut = (float)KDE_XCUT;  // FP32 packed kernels: truncation cut exponent (kde_fp32_cut)
};

#define KDE_ES_FROM_BOUND (-100000)

// exponent es of the fixed-point scale kde_acc_scale(bound) = 2^es
__device__ __forceinline__ int acc_scale_exp(double bound)
{
    int e;
    frexp(bound > 0 ? bound : 1.0, &e);
    return 62 - e;
}

// x 2^es rounded to the nearest integer, ties to even, in integer arithmetic: for
// -100 <= es <= 100 the same value as __double2ll_rn((double)x * 2^es) (the product
// is exact in FP64), without touching the FP64 pipe, which is slow on this part.
// |x| 2^es must stay below 2^62 (the scale's bound guarantees it).
__device__ __forceinline__ long long fix_pow2(float x, int es)
{
    const uint32_t b = __float_as_uint(x);
    const int be = (int)((b >> 23) & 0xffu);
    if (be == 0) return 0;  // zero or subnormal: |x| 2^es < 2^-126 2^100 < 1/2
    const int ex = be - 150 + es;  // |x| 2^es = m 2^ex with the 24-bit significand m
    const uint32_t m = (b & 0x7fffffu) | 0x800000u;
    long long q;
    if (ex >= 0) {
        q = (long long)m << (ex < 39 ? ex : 39);
    } else if (ex < -24) {
        q = 0;  // below 1/2
    } else {
        const int sh = -ex;  // 1 .. 24
        const uint32_t qq = m >> sh, rem = m & ((1u << sh) - 1u), half = 1u << (sh - 1);
        q = (long long)(qq + ((rem > half || (rem == half && (qq & 1u))) ? 1u : 0u));
    }
    return (b >> 31) ? -q : q;
}

__device__ __forceinline__ int window_nodes_f(float kappa, int Ng, float xcut)
{
    float s2 = xcut * (float)(KDE_LN2 / 2.0) / kappa;
    if (s2 >= 1.0f) return Ng;
    float r = 2.0f * asinf(sqrtf(s2));
    int w = (int)ceilf(r * (float)Ng * (float)(1.0 / KDE_TWO_PI)) + 1;
    return w >= Ng ? Ng : w;
}

template <typename T>
__device__ __forceinline__ void node_sc(const DepSrc<T> &S, int g, T &s, T &c)
{
    if (S.nodes) {
        typename V2<T>::t v = S.nodes[g];
        s = v.x;
        c = v.y;
    } else {
        // power-of-two grid: g / Ng is exact
        float sf, cf;
        sincospif((float)g / (float)S.Ng, &sf, &cf);
        s = sf;
        c = cf;
    }
}

template <typename T, bool UNSORTED = false>
__device__ void deposit_chunk_body(const DepSrc<T> &S, int64_t chunk, DepRec<T> *rec, T *part, int *red,
                                   int *cmm = nullptr)
{
    const int64_t i0 = chunk * DEP_CHUNK;
    if (i0 >= S.N) return;
    const int n = (int)(S.N - i0 < DEP_CHUNK ? S.N - i0 : DEP_CHUNK);
    const int Ng = S.Ng;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    int wloc = 0;
    int cmin = 0x7fffffff, cmax = -1;
    for (int t = tid; t < n; t += DEP_THREADS) {
        int64_t j = i0 + t;
        uint32_t uu = S.u[j];
        if (UNSORTED) {
            int cc = kde_cell(uu, S.Ng);
            cmin = cc < cmin ? cc : cmin;
            cmax = cc > cmax ? cc : cmax;
        }
        T k = S.kappa ? S.kscale * S.kappa[j] : S.kappa_u;
        if (!(k > (T)0 && k <= (T)KDE_KAPPA_MAX)) {
            kde_flag(S.status, KDE_DEV_KAPPA_RANGE, (unsigned)j);
            k = (T)KDE_KAPPA_MAX;
        }
        T nm;
        if (S.lnorm) nm = (T)exp2f(S.lnorm[j]);
        else if (S.norm) nm = S.norm[j];
        else if (S.kappa) nm = (T)kde_norm((double)k);
        else nm = S.norm_u;
        T wj = S.w ? S.w[j] : S.w_u;
        T sh, ch;
        kde_half_sincos(uu, sh, ch);
        T beta = sqrt((T)(2.0 * KDE_LOG2E) * k);
        rec[t].bs = beta * sh;
        rec[t].bc = beta * ch;
        rec[t].wn = wj * S.coef * nm;
        int wn_ = window_nodes_f((float)k, Ng, (float)KdeCut<T>::x);
        wloc = wn_ > wloc ? wn_ : wloc;
    }
    // block maximum of the window
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        int v = __shfl_xor_sync(0xffffffffu, wloc, o);
        wloc = v > wloc ? v : wloc;
    }
    if (lane == 0) red[warp] = wloc;
    __syncthreads();
    int W = 0;
#pragma unroll
    for (int k = 0; k < DEP_WARPS; ++k) W = red[k] > W ? red[k] : W;
    int c_first, c_last;
    if (UNSORTED) {
        // particles in any order: the chunk's linear cell range (a range that wraps
        // around the grid falls back to the whole grid below)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cmin = min(cmin, __shfl_xor_sync(0xffffffffu, cmin, o));
            cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
        }
        if (lane == 0) {
            cmm[warp] = cmin;
            cmm[DEP_WARPS + warp] = cmax;
        }
        __syncthreads();
        c_first = cmm[0];
        c_last = cmm[DEP_WARPS];
#pragma unroll
        for (int k = 1; k < DEP_WARPS; ++k) {
            c_first = min(c_first, cmm[k]);
            c_last = max(c_last, cmm[DEP_WARPS + k]);
        }
    } else {
        c_first = kde_cell(S.u[i0], Ng);
        c_last = kde_cell(S.u[i0 + n - 1], Ng);
    }
    int g_lo = c_first - W;
    int R = c_last + W - g_lo + 1;
    if (R >= Ng || c_last < c_first) {
        g_lo = 0;
        R = Ng;
    }
    const int ngroups = (R + 31) >> 5;

    double bound = S.bound;
    if (S.wmax_bits) bound = (double)S.N * (double)S.coef * S.norm_bound * (double)__uint_as_float(*S.wmax_bits);
    const double scale = kde_acc_scale(bound);

    if (ngroups >= DEP_WARPS) {
        for (int gi = warp; gi < ngroups; gi += DEP_WARPS) {
            int r = gi * 32 + lane;
            int g = g_lo + r;
            g = g < 0 ? g + Ng : (g >= Ng ? g - Ng : g);
            T Sg, Cg;
            node_sc(S, r < R ? g : 0, Sg, Cg);
            T acc = 0;
#pragma unroll 4
            for (int p = 0; p < n; ++p) {
                DepRec<T> q = rec[p];
                T s = Sg * q.bc - Cg * q.bs;
                acc += kde_ex2(-s * s) * q.wn;
            }
            if (r < R) {
                long long v = __double2ll_rn((double)acc * scale);
                if (v) atomicAdd((unsigned long long *)&S.acc[g], (unsigned long long)v);
            }
        }
        return;
    }
    const int slices = DEP_WARPS / ngroups;
    const int gi = warp % ngroups, sl = warp / ngroups;
    if (sl < slices) {
        int p0 = (int)((int64_t)n * sl / slices), p1 = (int)((int64_t)n * (sl + 1) / slices);
        int r = gi * 32 + lane;
        int g = g_lo + r;
        g = g < 0 ? g + Ng : (g >= Ng ? g - Ng : g);
        T Sg, Cg;
        node_sc(S, r < R ? g : 0, Sg, Cg);
        T acc = 0;
#pragma unroll 4
        for (int p = p0; p < p1; ++p) {
            DepRec<T> q = rec[p];
            T s = Sg * q.bc - Cg * q.bs;
            acc += kde_ex2(-s * s) * q.wn;
        }
        part[sl * (DEP_WARPS * 32) + r] = acc;
    }
    __syncthreads();
    for (int r = tid; r < ngroups * 32; r += DEP_THREADS) {
        if (r >= R) continue;
        T acc = 0;
        for (int k = 0; k < slices; ++k) acc += part[k * (DEP_WARPS * 32) + r];
        int g = g_lo + r;
        g = g < 0 ? g + Ng : (g >= Ng ? g - Ng : g);
        long long v = __double2ll_rn((double)acc * scale);
        if (v) atomicAdd((unsigned long long *)&S.acc[g], (unsigned long long)v);
    }
}

// ---------------------------------------------------------------------------
// FP32 chunk body with packed pair arithmetic: each lane owns two nodes (a warp
// pass covers 64 consecutive nodes) and every particle record is staged
// pre-duplicated, so that one 128-bit and one 64-bit broadcast load feed the
// f32x2 multiply-adds of both nodes.  Same node range, slicing and fixed-order
// combination as the scalar body.  Two forms of the kernel value, chosen per
// chunk by its largest width:
//  * half-angle (any width): 2^-(S_g beta c_j - C_g beta s_j)^2 with (s, c) the sine
//    and cosine of half the angle; records (beta s, beta s, beta c, beta c) and
//    (w n, w n); four multiply-adds per pair;
//  * cosine (largest width <= KDE_COSFORM_KMAX, when allowed): 2^(K cos(x_j - x_g))
//    2^-K with K = kappa log2(e); records (K cos, K cos, K sin, K sin) of the full
//    angle and (w n 2^-K, w n 2^-K); three multiply-adds per pair.
// ---------------------------------------------------------------------------
#define DEP2_PART 512
#define DEP2_UNROLL_P1 4
#define DEP2_UNROLL_P2 8

// node phase of the packed deposit: each lane owns P pairs of nodes, so a warp pass
// covers 64 P consecutive nodes of the chunk's range [g_lo, g_lo + R); with fewer
// groups than warps the warps split the particles into slices whose partial sums
// are combined in a fixed order
template <int P>
__device__ __forceinline__ void dep2_nodes(const DepSrc<float> &S, int n, int g_lo, int R, bool cosf, int es,
                                           const float4 *rsc, const float2 *rwn, float *part)
{
    constexpr int GW = 64 * P;
    constexpr int U = P == 2 ? DEP2_UNROLL_P2 : DEP2_UNROLL_P1;  // particle loop unrolling
    const int Ng = S.Ng;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ngroups = (R + GW - 1) / GW;
    const bool fix_int = es >= -100 && es <= 100;
    // the FP64 conversion, for extreme bounds only; 2^es built from its bits
    const double scale = __longlong_as_double((long long)(1023 + (es < -1000 ? -1000 : (es > 1000 ? 1000 : es))) << 52);

    int gn[2 * P];
    bool ok[2 * P];
    kde_f2 SS[P], CC[P], acc[P];
    auto nodes_of = [&](int gi) {
#pragma unroll
        for (int m = 0; m < 2 * P; ++m) {
            const int r = gi * GW + m * 32 + lane;
            ok[m] = r < R;
            int g = g_lo + r;
            g = g < 0 ? g + Ng : (g >= Ng ? g - Ng : g);
            gn[m] = g;
        }
#pragma unroll
        for (int q = 0; q < P; ++q) {
            float sa, ca, sb, cb;
            node_sc(S, ok[2 * q] ? gn[2 * q] : 0, sa, ca);
            node_sc(S, ok[2 * q + 1] ? gn[2 * q + 1] : 0, sb, cb);
            if (cosf) {
                // sine and cosine of the full node angle
                SS[q] = kde_pk(2.f * sa * ca, 2.f * sb * cb);
                CC[q] = kde_pk((ca - sa) * (ca + sa), (cb - sb) * (cb + sb));
            } else {
                SS[q] = kde_pk(sa, sb);
                CC[q] = kde_pk(-ca, -cb);
            }
        }
    };
    auto sweep = [&](int p0, int p1) {
#pragma unroll
        for (int q = 0; q < P; ++q) acc[q] = kde_pk(0.f, 0.f);
        if (cosf) {
#pragma unroll U
            for (int p = p0; p < p1; ++p) {
                const float4 r4 = rsc[p];
                const float2 w2 = rwn[p];
                const kde_f2 qs = kde_pk(r4.z, r4.w), qc = kde_pk(r4.x, r4.y), w = kde_pk(w2.x, w2.y);
                // K cos(x_j - x_g) = sin_g (K sin_j) + cos_g (K cos_j)
#pragma unroll
                for (int q = 0; q < P; ++q)
                    acc[q] = kde_fma2(kde_ex22(kde_fma2(SS[q], qs, kde_mul2(CC[q], qc))), w, acc[q]);
            }
        } else {
#pragma unroll U
            for (int p = p0; p < p1; ++p) {
                const float4 r4 = rsc[p];
                const float2 w2 = rwn[p];
                const kde_f2 qs = kde_pk(r4.z, r4.w), qc = kde_pk(r4.x, r4.y), w = kde_pk(w2.x, w2.y);
                // s = S_g (beta cos_j) - C_g (beta sin_j)
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const kde_f2 sv = kde_fma2(SS[q], qs, kde_mul2(CC[q], qc));
                    acc[q] = kde_fma2(kde_ex2neg2(kde_mul2(sv, sv)), w, acc[q]);
                }
            }
        }
    };
    auto fix = [&](float a) -> long long { return fix_int ? fix_pow2(a, es) : __double2ll_rn((double)a * scale); };

    if (ngroups >= DEP_WARPS) {
        for (int gi = warp; gi < ngroups; gi += DEP_WARPS) {
            nodes_of(gi);
            sweep(0, n);
#pragma unroll
            for (int q = 0; q < P; ++q) {
                float a0, a1;
                kde_upk(acc[q], a0, a1);
                long long v;
                if (ok[2 * q] && (v = fix(a0)) != 0) atomicAdd((unsigned long long *)&S.acc[gn[2 * q]], (unsigned long long)v);
                if (ok[2 * q + 1] && (v = fix(a1)) != 0)
                    atomicAdd((unsigned long long *)&S.acc[gn[2 * q + 1]], (unsigned long long)v);
            }
        }
        return;
    }
    // every warp works: warp w takes node group w mod ngroups and one of that group's
    // particle slices (the groups' slice counts differ by at most one); ngroups GW <= DEP2_PART
    const int gi = warp % ngroups, sl = warp / ngroups;
    const int slices = (DEP_WARPS - gi + ngroups - 1) / ngroups;
    {
        const int p0 = (int)((int64_t)n * sl / slices), p1 = (int)((int64_t)n * (sl + 1) / slices);
        nodes_of(gi);
        sweep(p0, p1);
#pragma unroll
        for (int q = 0; q < P; ++q) {
            float a0, a1;
            kde_upk(acc[q], a0, a1);
            part[sl * DEP2_PART + gi * GW + 64 * q + lane] = a0;
            part[sl * DEP2_PART + gi * GW + 64 * q + 32 + lane] = a1;
        }
    }
    __syncthreads();
    for (int r = tid; r < ngroups * GW; r += DEP_THREADS) {
        if (r >= R) continue;
        const int gr = r / GW, sr = (DEP_WARPS - gr + ngroups - 1) / ngroups;
        float a = 0.f;
        for (int k = 0; k < sr; ++k) a += part[k * DEP2_PART + r];
        int g = g_lo + r;
        g = g < 0 ? g + Ng : (g >= Ng ? g - Ng : g);
        const long long v = fix(a);
        if (v) atomicAdd((unsigned long long *)&S.acc[g], (unsigned long long)v);
    }
}

__device__ void deposit_chunk_body_x2(const DepSrc<float> &S, int64_t chunk, float4 *rsc, float2 *rwn, float *part,
                                      int *red, bool allow_cos)
{
    const int64_t i0 = chunk * DEP_CHUNK;
    if (i0 >= S.N) return;
    const int n = (int)(S.N - i0 < DEP_CHUNK ? S.N - i0 : DEP_CHUNK);
    const int Ng = S.Ng;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // every input of the thread's particles loaded at once (one global-load latency per
    // chunk); the smallest width sets the window, the largest the form
    constexpr int PER = DEP_CHUNK / DEP_THREADS;
    uint32_t ru[PER];
    float rk[PER], rn[PER], rw[PER];
    float kmin = (float)KDE_KAPPA_MAX, kmax = 0.f;
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int t = tid + p * DEP_THREADS;
        const bool ok = t < n;
        const int64_t j = i0 + (ok ? t : 0);
        ru[p] = S.u[j];
        float k = S.kappa ? S.kscale * S.kappa[j] : S.kappa_u;
        rn[p] = S.lnorm ? S.lnorm[j] : (S.norm ? S.norm[j] : 0.f);
        rw[p] = S.w ? S.w[j] : S.w_u;
        if (ok && !(k > 0.f && k <= (float)KDE_KAPPA_MAX)) {
            kde_flag(S.status, KDE_DEV_KAPPA_RANGE, (unsigned)j);
            k = (float)KDE_KAPPA_MAX;
        }
        rk[p] = k;
        if (ok) {
            kmin = fminf(kmin, k);
            kmax = fmaxf(kmax, k);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kmin = fminf(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
        kmax = fmaxf(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    }
    if (lane == 0) {
        red[warp] = __float_as_int(kmin);
        red[DEP_WARPS + warp] = __float_as_int(kmax);
    }
    // the fixed-point scale 2^es, worked out by one thread: FP64 stays off the other threads
    __shared__ int s_es;
    if (tid == 0) {
        int es = S.scale_exp;
        if (es == KDE_ES_FROM_BOUND) {
            double bound = S.bound;
            if (S.wmax_bits)
                bound = (double)S.N * (double)S.coef * S.norm_bound * (double)__uint_as_float(*S.wmax_bits);
            es = acc_scale_exp(bound);
        }
        s_es = es;
    }
    __syncthreads();
    const int es = s_es;
#pragma unroll
    for (int k = 0; k < DEP_WARPS; ++k) {
        kmin = fminf(kmin, __int_as_float(red[k]));
        kmax = fmaxf(kmax, __int_as_float(red[DEP_WARPS + k]));
    }
    // the window shrinks as the width grows: the smallest width's window covers all
    const int W = window_nodes_f(kmin, Ng, S.xcut);
    const bool cosf = allow_cos && kmax <= KDE_COSFORM_KMAX;
    // the particle records
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int t = tid + p * DEP_THREADS;
        if (t >= n) break;
        const uint32_t uu = ru[p];
        const float k = rk[p];
        float nm;
        if (S.lnorm) nm = exp2f(rn[p]);
        else if (S.norm) nm = rn[p];
        else if (S.kappa) nm = S.ntab ? kde_norm_tab(S.ntab, k) : (float)kde_norm((double)k);
        else nm = S.norm_u;
        const float wn = rw[p] * S.coef * nm;
        float sh, ch;
        kde_half_sincos(uu, sh, ch);
        if (cosf) {
            const float K = (float)KDE_LOG2E * k;
            const float cx = (ch - sh) * (ch + sh), sx = 2.f * sh * ch;
            rsc[t] = make_float4(K * cx, K * cx, K * sx, K * sx);
            const float wk = wn * kde_ex2(-K);
            rwn[t] = make_float2(wk, wk);
        } else {
            const float beta = sqrtf((float)(2.0 * KDE_LOG2E) * k);
            rsc[t] = make_float4(beta * sh, beta * sh, beta * ch, beta * ch);
            rwn[t] = make_float2(wn, wn);
        }
    }
    __syncthreads();
    const int c_first = kde_cell(S.u[i0], Ng), c_last = kde_cell(S.u[i0 + n - 1], Ng);
    int g_lo = c_first - W;
    int R = c_last + W - g_lo + 1;
    if (R >= Ng || R < 1 || c_last < c_first) {
        g_lo = 0;
        R = Ng;
    }
    // two node pairs a lane halve the particle loads per pair: taken where the wider
    // groups compute no extra nodes and their partial sums fit the buffer
    const int n64 = (R + 63) >> 6, n128 = (R + 127) >> 7;
    if (2 * n128 == n64 && (n128 >= DEP_WARPS || n128 * 128 <= DEP2_PART))
        dep2_nodes<2>(S, n, g_lo, R, cosf, es, rsc, rwn, part);
    else
        dep2_nodes<1>(S, n, g_lo, R, cosf, es, rsc, rwn, part);
}

__global__ void __launch_bounds__(DEP_THREADS) deposit_chunk_x2_kernel(DepSrc<float> S)
{
    __shared__ float4 rsc[DEP_CHUNK];
    __shared__ float2 rwn[DEP_CHUNK];
    __shared__ float part[DEP_WARPS * DEP2_PART];
    __shared__ int red[2 * DEP_WARPS];
    deposit_chunk_body_x2(S, blockIdx.x, rsc, rwn, part, red, true);
}

template <typename T>
__global__ void __launch_bounds__(DEP_THREADS) deposit_chunk_kernel(DepSrc<T> S)
{
    __shared__ DepRec<T> rec[DEP_CHUNK];
    __shared__ T part[DEP_WARPS * 32 * DEP_WARPS];
    __shared__ int red[DEP_WARPS];
    deposit_chunk_body<T>(S, blockIdx.x, rec, part, red);
}

// ---------------------------------------------------------------------------
// FP32 deposit of cell-sorted particles over a balanced persistent grid, without
// global atomics.
//
// G = min(3 x SMs, ceil(N / 256)) CTAs (one wave); CTA c owns the contiguous
// particles [c N / G, (c + 1) N / G), so every CTA carries the same number of
// particles and, since a particle's cost is its window, nearly the same work.
// The CTA's node window is fixed up front: its first and last cell widened by the
// window of its smallest width.  Its particles are taken in sub-chunks of
// DEPP_SUB records (one float4 each: the two angle terms and the weighted norm;
// a Landau-size run of 2^20 particles has one sub-chunk a CTA), the inputs of a
// sub-chunk loaded in batches of register loads, and swept by node-owner lanes as
// in the chunk kernel (f32x2 pairs of nodes, fixed-order combination of particle
// slices).  After every sub-chunk the FP32 node sums become int64 fixed point in
// the CTA's row of the workspace (each node always by the same thread: plain
// loads and stores).  A second kernel sums the rows: one CTA per 32 nodes, its
// warps taking the rows in turn with all their loads in flight, the warps'
// integer sums combined in shared memory, every output node written with a plain
// store.  Integer sums make the result exact and independent of any order.
// ---------------------------------------------------------------------------
#define DEPP_THREADS 256
#define DEPP_WARPS 8
#define DEPP_MINB 3  // CTAs an SM (80 registers a thread): 7% faster than 4 at 64 registers
#define DEPP_SUB 2304  // records a sub-chunk: a 2^20-particle run has one sub-chunk a CTA
#define DEPP_PART 512
#define DEPP_RED_THREADS 1024
#define DEPP_RED_NODES 32

struct DepPlan {
    int G;            // CTAs
    long long *rows;  // [G][Ng] per-CTA node sums over its window
    int2 *hdr;        // [G] (first node, node count) of every row
    long long *acc;   // [Ng] output accumulators (every node written by the row reduction)
};
// node pairs of the persistent deposit: each lane owns P pairs of nodes (64 P
// consecutive nodes a warp pass) of the window [g_lo, g_lo + R); the n records of
// the sub-chunk are split into slices when there are fewer node groups than warps.
// flush(r, a) receives the FP32 sum of window node r over the sub-chunk, once per node.
template <int P, typename F>
__device__ __forceinline__ void depp_sweep(const DepSrc<float> &S, int n, int g_lo, int R, bool cosf,
                                           const float4 *rec, float *part, F &&flush)
{
    constexpr int GW = 64 * P;
    constexpr int U = 4;
    const int Ng = S.Ng;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ngroups = (R + GW - 1) / GW;
    kde_f2 SS[P], CC[P], acc[P];
    auto nodes_of = [&](int gi) {
#pragma unroll
        for (int q = 0; q < P; ++q) {
            float sa, ca, sb, cb;
            const int ra = gi * GW + 64 * q + lane, rb = ra + 32;
            int ga = g_lo + ra, gb = g_lo + rb;
            ga = ga < 0 ? ga + Ng : (ga >= Ng ? ga - Ng : ga);
            gb = gb < 0 ? gb + Ng : (gb >= Ng ? gb - Ng : gb);
            node_sc(S, ra < R ? ga : 0, sa, ca);
            node_sc(S, rb < R ? gb : 0, sb, cb);
            if (cosf) {
                SS[q] = kde_pk(2.f * sa * ca, 2.f * sb * cb);
                CC[q] = kde_pk((ca - sa) * (ca + sa), (cb - sb) * (cb + sb));
            } else {
                SS[q] = kde_pk(sa, sb);
                CC[q] = kde_pk(-ca, -cb);
            }
        }
    };
    // record (a, b, w): cosine form a = K cos x_j, b = K sin x_j, exponent
    // S_g b + C_g a = K cos(x_j - x_g); half-angle form a = beta sin, b = beta cos of
    // half the angle, s = S_g b - C_g a and the exponent -s^2
    auto sweep = [&](int p0, int p1) {
#pragma unroll
        for (int q = 0; q < P; ++q) acc[q] = kde_pk(0.f, 0.f);
        if (cosf) {
#pragma unroll U
            for (int p = p0; p < p1; ++p) {
                const float4 r4 = rec[p];
                const kde_f2 qa = kde_pk(r4.x, r4.x), qb = kde_pk(r4.y, r4.y), w = kde_pk(r4.z, r4.z);
#pragma unroll
                for (int q = 0; q < P; ++q)
                    acc[q] = kde_fma2(kde_ex22(kde_fma2(SS[q], qb, kde_mul2(CC[q], qa))), w, acc[q]);
            }
        } else {
#pragma unroll U
            for (int p = p0; p < p1; ++p) {
                const float4 r4 = rec[p];
                const kde_f2 qa = kde_pk(r4.x, r4.x), qb = kde_pk(r4.y, r4.y), w = kde_pk(r4.z, r4.z);
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const kde_f2 sv = kde_fma2(SS[q], qb, kde_mul2(CC[q], qa));
                    acc[q] = kde_fma2(kde_ex2neg2(kde_mul2(sv, sv)), w, acc[q]);
                }
            }
        }
    };
    if (ngroups >= DEPP_WARPS) {
        for (int gi = warp; gi < ngroups; gi += DEPP_WARPS) {
            nodes_of(gi);
            sweep(0, n);
#pragma unroll
            for (int q = 0; q < P; ++q) {
                float a0, a1;
                kde_upk(acc[q], a0, a1);
                const int ra = gi * GW + 64 * q + lane;
                if (ra < R) flush(ra, a0);
                if (ra + 32 < R) flush(ra + 32, a1);
            }
        }
        return;
    }
    // every warp works: warp w takes node group w mod ngroups and one of that group's
    // particle slices (slice counts differ by at most one); ngroups GW <= DEPP_PART
    const int gi = warp % ngroups, sl = warp / ngroups;
    const int slices = (DEPP_WARPS - gi + ngroups - 1) / ngroups;
    {
        const int p0 = (int)((int64_t)n * sl / slices), p1 = (int)((int64_t)n * (sl + 1) / slices);
        nodes_of(gi);
        sweep(p0, p1);
#pragma unroll
        for (int q = 0; q < P; ++q) {
            float a0, a1;
            kde_upk(acc[q], a0, a1);
            part[sl * DEPP_PART + gi * GW + 64 * q + lane] = a0;
            part[sl * DEPP_PART + gi * GW + 64 * q + 32 + lane] = a1;
        }
    }
    __syncthreads();
    for (int r = tid; r < ngroups * GW; r += DEPP_THREADS) {
        if (r >= R) continue;
        const int gr = r / GW, sr = (DEPP_WARPS - gr + ngroups - 1) / ngroups;
        float a = 0.f;
        for (int k = 0; k < sr; ++k) a += part[k * DEPP_PART + r];
        flush(r, a);
    }
}

// narrow windows (R <= 32 NPL nodes): the records are kept in particle pairs, recAB[k] =
// (a_2k, a_2k+1, b_2k, b_2k+1) and recW[k] = (w_2k, w_2k+1), so that one packed operation
// serves two particles of the same node.  A lane owns NPL nodes (j, j + LG, ...) of its
// group of LG lanes; the 32 / LG groups of a warp (slices) and the eight warps take
// interleaved particle pairs.  Slice sums are combined by a fixed butterfly over the lane
// bits above LG, warp sums in warp order; flush(r, a) receives each node's sum once.
template <int LG, int NPL, typename F>
__device__ __forceinline__ void depp_sweep_pairs(const DepSrc<float> &S, int n, int g_lo, int R, bool cosf,
                                                 const float4 *recAB, const float2 *recW, float *part, F &&flush)
{
    constexpr int SL = 32 / LG;
    constexpr int U = 4;
    const int Ng = S.Ng;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int j = lane & (LG - 1), sl = lane / LG;
    kde_f2 SS[NPL], CC[NPL], acc[NPL];
#pragma unroll
    for (int t = 0; t < NPL; ++t) {
        const int r = j + LG * t;
        int g = g_lo + r;
        g = g < 0 ? g + Ng : (g >= Ng ? g - Ng : g);
        float sg, cg;
        node_sc(S, r < R ? g : 0, sg, cg);
        if (cosf) {
            const float sf = 2.f * sg * cg, cf = (cg - sg) * (cg + sg);
            SS[t] = kde_pk(sf, sf);
            CC[t] = kde_pk(cf, cf);
        } else {
            SS[t] = kde_pk(sg, sg);
            CC[t] = kde_pk(-cg, -cg);
        }
        acc[t] = kde_pk(0.f, 0.f);
    }
    const int np = (n + 1) >> 1;
    const int k0 = (int)((int64_t)np * warp / DEPP_WARPS), k1 = (int)((int64_t)np * (warp + 1) / DEPP_WARPS);
    if (cosf) {
#pragma unroll U
        for (int k = k0 + sl; k < k1; k += SL) {
            const float4 ab = recAB[k];
            const float2 w = recW[k];
            const kde_f2 A = kde_pk(ab.x, ab.y), B = kde_pk(ab.z, ab.w), W2 = kde_pk(w.x, w.y);
#pragma unroll
            for (int t = 0; t < NPL; ++t) acc[t] = kde_fma2(kde_ex22(kde_fma2(SS[t], B, kde_mul2(CC[t], A))), W2, acc[t]);
        }
    } else {
#pragma unroll U
        for (int k = k0 + sl; k < k1; k += SL) {
            const float4 ab = recAB[k];
            const float2 w = recW[k];
            const kde_f2 A = kde_pk(ab.x, ab.y), B = kde_pk(ab.z, ab.w), W2 = kde_pk(w.x, w.y);
#pragma unroll
            for (int t = 0; t < NPL; ++t) {
                const kde_f2 sv = kde_fma2(SS[t], B, kde_mul2(CC[t], A));
                acc[t] = kde_fma2(kde_ex2neg2(kde_mul2(sv, sv)), W2, acc[t]);
            }
        }
    }
#pragma unroll
    for (int t = 0; t < NPL; ++t) {
        float a0, a1;
        kde_upk(acc[t], a0, a1);
        float a = a0 + a1;
#pragma unroll
        for (int o = LG; o < 32; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (sl == 0) part[warp * DEPP_PART + j + LG * t] = a;
    }
    __syncthreads();
    for (int r = tid; r < R; r += DEPP_THREADS) {
        float a = 0.f;
#pragma unroll
        for (int w = 0; w < DEPP_WARPS; ++w) a += part[w * DEPP_PART + r];
        flush(r, a);
    }
}

// acc[g] = sum over the rows whose window covers node g of that row's entry; CTA b
// takes nodes [32 b, 32 b + 32), lane l node 32 b + l, warp w rows w, w + 32, ...
__global__ void __launch_bounds__(DEPP_RED_THREADS) deposit_rows_kernel(const long long *__restrict__ rows,
                                                                       const int2 *__restrict__ hdr, int G, int Ng,
                                                                       long long *acc)
{
    __shared__ long long wsum[DEPP_RED_THREADS / 32][DEPP_RED_NODES];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = DEPP_RED_THREADS / 32;
    const int g = blockIdx.x * DEPP_RED_NODES + lane;
    long long sum = 0;
    if (g < Ng) {
        // rows in batches of 8 per warp, every load of a batch issued before any is used
        for (int k0 = warp; k0 < G; k0 += 8 * NW) {
            long long v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = k0 + q * NW;
                v[q] = 0;
                if (k < G) {
                    const int2 h = hdr[k];
                    int r = g - h.x;
                    r = r < 0 ? r + Ng : (r >= Ng ? r - Ng : r);
                    if (r < h.y) v[q] = rows[(size_t)k * Ng + r];
                }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) sum += v[q];
        }
    }
    wsum[warp][lane] = sum;
    __syncthreads();
    if (warp == 0 && g < Ng) {
        long long t = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) t += wsum[w][lane];
        acc[g] = t;
    }
}

__global__ void __launch_bounds__(DEPP_THREADS, DEPP_MINB) deposit_persist_kernel(DepSrc<float> S, DepPlan Pl)
{
    __shared__ float4 rec[DEPP_SUB];
    __shared__ float part[DEPP_WARPS * DEPP_PART];
    __shared__ float sred[2 * DEPP_WARPS];
    __shared__ int s_es;
    constexpr int PER = DEPP_SUB / DEPP_THREADS;  // particles of a sub-chunk per thread
    const int Ng = S.Ng;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c = blockIdx.x;
    const int64_t i0 = S.N * c / Pl.G, i1 = S.N * (c + 1) / Pl.G;  // non-empty: G <= N
    kde_pdl_wait();  // everything read below comes from the sort before
    kde_pdl_trigger();

    // smallest and largest width of the CTA's particles (the window and the form): a pass
    // over the widths, PER loads in flight per thread
    float kmin = (float)KDE_KAPPA_MAX, kmax = 0.f;
    for (int64_t j0 = i0; j0 < i1; j0 += (int64_t)PER * DEPP_THREADS) {
        float kk[PER];
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            const int64_t j = j0 + tid + p * DEPP_THREADS;
            kk[p] = j < i1 ? (S.kappa ? S.kscale * S.kappa[j] : S.kappa_u) : -1.f;
        }
#pragma unroll
        for (int p = 0; p < PER; ++p)
            if (kk[p] != -1.f) {
                const float k = (kk[p] > 0.f && kk[p] <= (float)KDE_KAPPA_MAX) ? kk[p] : (float)KDE_KAPPA_MAX;
                kmin = fminf(kmin, k);
                kmax = fmaxf(kmax, k);
            }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kmin = fminf(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
        kmax = fmaxf(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    }
    if (lane == 0) {
        sred[warp] = kmin;
        sred[DEPP_WARPS + warp] = kmax;
    }
    if (tid == 0) {
        int es = S.scale_exp;
        if (es == KDE_ES_FROM_BOUND) {
            double bound = S.bound;
            if (S.wmax_bits)
                bound = (double)S.N * (double)S.coef * S.norm_bound * (double)__uint_as_float(*S.wmax_bits);
            es = acc_scale_exp(bound);
        }
        s_es = es;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < DEPP_WARPS; ++k) {
        kmin = fminf(kmin, sred[k]);
        kmax = fmaxf(kmax, sred[DEPP_WARPS + k]);
    }
    const int es = s_es;
    const bool cosf = kmax <= KDE_COSFORM_KMAX;
    const int W = window_nodes_f(kmin, Ng, S.xcut);
    const int c_first = kde_cell(S.u[i0], Ng), c_last = kde_cell(S.u[i1 - 1], Ng);
    int g_lo = c_first - W;
    int R = c_last + W - g_lo + 1;
    if (R >= Ng || R < 1 || c_last < c_first) {
        g_lo = 0;
        R = Ng;
    }
    // windows of up to 128 nodes: records in particle pairs (depp_sweep_pairs); wider ones:
    // 4, 2 or 1 node pairs a lane, the widest that computes no extra nodes and whose slice
    // sums fit the buffer
    const bool pairs = R <= 128;
    float4 *recAB = rec;
    float2 *recW = (float2 *)(rec + DEPP_SUB / 2);
    const int n64 = (R + 63) >> 6, n128 = (R + 127) >> 7, n256 = (R + 255) >> 8;
    const int P = (4 * n256 == n64 && (n256 >= DEPP_WARPS || n256 * 256 <= DEPP_PART))   ? 4
                  : (2 * n128 == n64 && (n128 >= DEPP_WARPS || n128 * 128 <= DEPP_PART)) ? 2
                                                                                          : 1;
    long long *row = Pl.rows + (size_t)c * Ng;

    for (int64_t b0 = i0; b0 < i1; b0 += DEPP_SUB) {
        const int n = (int)(i1 - b0 < DEPP_SUB ? i1 - b0 : DEPP_SUB);
        const bool first = b0 == i0;
        if (!first) __syncthreads();  // the previous sub-chunk's readers of rec and part are done
        // the particle records (a, b, w n) of the form in use, in groups of four particles a
        // thread whose inputs are loaded together (one global-load latency per group)
        constexpr int QB = 4;
#pragma unroll 1
        for (int p0 = 0; p0 < PER; p0 += QB) {
            uint32_t ru[QB];
            float rk[QB], rn[QB], rw[QB];
#pragma unroll
            for (int q = 0; q < QB; ++q) {
                const int t = tid + (p0 + q) * DEPP_THREADS;
                const int64_t j = b0 + (t < n ? t : 0);
                ru[q] = S.u[j];
                rk[q] = S.kappa ? S.kscale * S.kappa[j] : S.kappa_u;
                rn[q] = S.norm ? S.norm[j] : 0.f;
                rw[q] = S.w ? S.w[j] : S.w_u;
            }
#pragma unroll
            for (int q = 0; q < QB; ++q) {
                const int t = tid + (p0 + q) * DEPP_THREADS;
                if (t >= n) break;
                float k = rk[q];
                if (!(k > 0.f && k <= (float)KDE_KAPPA_MAX)) {
                    kde_flag(S.status, KDE_DEV_KAPPA_RANGE, (unsigned)(b0 + t));
                    k = (float)KDE_KAPPA_MAX;
                }
                float nm;
                if (S.norm) nm = rn[q];
                else if (S.kappa) nm = S.ntab ? kde_norm_tab(S.ntab, k) : (float)kde_norm((double)k);
                else nm = S.norm_u;
                const float wn = rw[q] * S.coef * nm;
                float sh, ch;
                kde_half_sincos(ru[q], sh, ch);
                float ra, rb, rw2;
                if (cosf) {
                    const float K = (float)KDE_LOG2E * k;
                    ra = K * ((ch - sh) * (ch + sh));
                    rb = K * (2.f * sh * ch);
                    rw2 = wn * kde_ex2(-K);
                } else {
                    const float beta = sqrtf((float)(2.0 * KDE_LOG2E) * k);
                    ra = beta * sh;
                    rb = beta * ch;
                    rw2 = wn;
                }
                if (pairs) {
                    float *ab = (float *)recAB + (t >> 1) * 4 + (t & 1);
                    ab[0] = ra;
                    ab[2] = rb;
                    ((float *)recW)[t] = rw2;
                } else {
                    rec[t] = make_float4(ra, rb, rw2, 0.f);
                }
            }
        }
        if (pairs && (n & 1) && tid == 0) {
            // the odd particle's partner: no weight (a finite exponent times zero)
            float *ab = (float *)recAB + (n >> 1) * 4 + 1;
            ab[0] = 0.f;
            ab[2] = 0.f;
            ((float *)recW)[n] = 0.f;
        }
        __syncthreads();
        auto flush = [&](int r, float a) {
            // x 2^es in integer arithmetic; the FP64 product only for extreme bounds
            const long long v = (es >= -100 && es <= 100) ? fix_pow2(a, es) : __double2ll_rn(ldexp((double)a, es));
            row[r] = first ? v : __ldcg(&row[r]) + v;
        };
        if (pairs) {
            if (R <= 8) depp_sweep_pairs<8, 1>(S, n, g_lo, R, cosf, recAB, recW, part, flush);
            else if (R <= 16) depp_sweep_pairs<16, 1>(S, n, g_lo, R, cosf, recAB, recW, part, flush);
            else if (R <= 32) depp_sweep_pairs<32, 1>(S, n, g_lo, R, cosf, recAB, recW, part, flush);
            else if (R <= 64) depp_sweep_pairs<32, 2>(S, n, g_lo, R, cosf, recAB, recW, part, flush);
            else depp_sweep_pairs<32, 4>(S, n, g_lo, R, cosf, recAB, recW, part, flush);
        } else if (P == 4) depp_sweep<4>(S, n, g_lo, R, cosf, rec, part, flush);
        else if (P == 2) depp_sweep<2>(S, n, g_lo, R, cosf, rec, part, flush);
        else depp_sweep<1>(S, n, g_lo, R, cosf, rec, part, flush);
    }
    if (tid == 0) Pl.hdr[c] = make_int2(g_lo, R);
}

// acc -> real values
template <typename T>
__global__ void acc_to_real_kernel(const long long *acc, int Ng, double bound, const unsigned int *wmax_bits,
                                   double wscale, T *out)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Ng) return;
    double b = wmax_bits ? wscale * (double)__uint_as_float(*wmax_bits) : bound;
    out[g] = (T)((double)acc[g] / kde_acc_scale(b));
}

// largest weight (non-negative floats order like their bit patterns)
template <typename T>
__global__ void wmax_kernel(const T *w, int64_t N, unsigned int *wmax_bits, unsigned int *status)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float m = 0.f;
    for (; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        float v = (float)w[i];
        if (!(v >= 0.f) || isinf(v)) kde_flag(status, KDE_DEV_BAD_ARG, (unsigned)i);
        else m = fmaxf(m, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    // round the maximum up by one ulp so that the float bound of a double weight still bounds it
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(wmax_bits, __float_as_uint(m) + 1u);
}

// ---------------------------------------------------------------------------
// workspace of the persistent FP32 deposit for N particles on Ng nodes: the CTAs'
// rows and their headers
static kde_status depp_plan(kde_ctx *ctx, int64_t N, int Ng, long long *acc, DepPlan &Pl)
{
    const int64_t gmax = (int64_t)DEPP_MINB * ctx->sm_count;
    const int64_t gn = (N + 255) / 256;
    Pl.G = (int)(gn < gmax ? gn : gmax);
    const size_t rows_b = (size_t)Pl.G * Ng * 8;
    unsigned char *w = (unsigned char *)kde_ws(ctx, WS_DEP_ROWS, rows_b + (size_t)Pl.G * 8);
    if (!w) return KDE_ENOMEM;
    Pl.rows = (long long *)w;
    Pl.hdr = (int2 *)(w + rows_b);
    Pl.acc = acc;
    return KDE_OK;
}

kde_status kde_deposit_reserve(kde_ctx *ctx, int64_t N, int Ng)
{
    DepPlan Pl{};
    return depp_plan(ctx, N, Ng, nullptr, Pl);
}

template <typename T>
static kde_status deposit_sorted_impl(kde_ctx *ctx, const uint32_t *u, const T *kappa, T kappa_u, const T *norm,
                                      T norm_u, const T *w, T w_u, int64_t N, int Ng, double coef, long long *acc,
                                      double bound, const unsigned int *wmax_bits, double norm_bound, DepRows *rows_out,
                                      float xcut = 0.f)
{
    // the persistent FP32 kernel writes every node; the others add into zeroed accumulators
    if (!(sizeof(T) == 4 && N > 0))
        KDE_CUDA(ctx, cudaMemsetAsync(acc, 0, (size_t)Ng * sizeof(long long), ctx->stream), "acc memset");
    if (N == 0) return KDE_OK;
    const void *nodes = kde_node_table(ctx, Ng, sizeof(T) == 8);
    if (!nodes) return KDE_ENOMEM;
    DepSrc<T> S{};
    S.u = u;
    S.N = N;
    S.kappa = kappa;
    S.kappa_u = kappa_u;
    S.kscale = (T)1;
    S.norm = norm;
    S.lnorm = nullptr;
    S.norm_u = norm_u;
    S.w = w;
    S.w_u = w_u;
    S.coef = (T)coef;
    S.Ng = Ng;
    S.nodes = (const typename V2<T>::t *)nodes;
    S.acc = acc;
    S.bound = bound;
    S.wmax_bits = wmax_bits;
    S.norm_bound = norm_bound;
    S.status = ctx->d_status;
    S.scale_exp = KDE_ES_FROM_BOUND;
    if (!wmax_bits) {
        // the scale exponent from the host-known bound, as acc_scale_exp computes it
        int e;
        frexp(bound > 0 ? bound : 1.0, &e);
        S.scale_exp = 62 - e;
    }
    S.ntab = ctx->norm_tab;
    S.xcut = xcut > 0.f ? xcut : kde_fp32_cut(ctx);
    if constexpr (sizeof(T) == 4) {
        DepPlan Pl{};
        KDE_TRY(depp_plan(ctx, N, Ng, acc, Pl));
        {
            KdeProfScope _ps(ctx, PROF_DEPOSIT);
            KDE_CUDA(ctx, kde_launch(ctx, true, deposit_persist_kernel, dim3(Pl.G), dim3(DEPP_THREADS), 0, S, Pl),
                     "deposit_persist_kernel");
        }
        KDE_LAUNCHED(ctx, "deposit_persist_kernel");
        if (rows_out) {
            // the caller sums the rows itself (the PIC step's field kernel)
            rows_out->rows = Pl.rows;
            rows_out->hdr = Pl.hdr;
            rows_out->G = Pl.G;
            return KDE_OK;
        }
        {
            KdeProfScope _ps(ctx, PROF_DEPOSIT_ROWS);
            deposit_rows_kernel<<<(Ng + DEPP_RED_NODES - 1) / DEPP_RED_NODES, DEPP_RED_THREADS, 0, ctx->stream>>>(
                Pl.rows, Pl.hdr, Pl.G, Ng, acc);
        }
        KDE_LAUNCHED(ctx, "deposit_rows_kernel");
    } else {
        unsigned grid = (unsigned)((N + DEP_CHUNK - 1) / DEP_CHUNK);
        {
            KdeProfScope _ps(ctx, PROF_DEPOSIT);
            deposit_chunk_kernel<T><<<grid, DEP_THREADS, 0, ctx->stream>>>(S);
        }
        KDE_LAUNCHED(ctx, "deposit_chunk_kernel");
    }
    return KDE_OK;
}

template <typename T>
kde_status kde_deposit_sorted(kde_ctx *ctx, const uint32_t *u, const T *kappa, T kappa_u, const T *norm, T norm_u,
                              const T *w, T w_u, int64_t N, int Ng, double coef, long long *acc, double bound,
                              const unsigned int *wmax_bits, double norm_bound)
{
    return deposit_sorted_impl<T>(ctx, u, kappa, kappa_u, norm, norm_u, w, w_u, N, Ng, coef, acc, bound, wmax_bits,
                                  norm_bound, nullptr);
}

kde_status kde_deposit_rows_f32(kde_ctx *ctx, const uint32_t *u, const float *kappa, float kappa_u, const float *norm,
                                float norm_u, int64_t N, int Ng, double coef, float w_u, double bound, DepRows *out,
                                float xcut)
{
    if (N < 1) return kde_fail(ctx, KDE_EINVAL, "deposit rows: need N >= 1");
    return deposit_sorted_impl<float>(ctx, u, kappa, kappa_u, norm, norm_u, nullptr, w_u, N, Ng, coef, nullptr, bound,
                                      nullptr, 0.0, out, xcut);
}

template <typename T>
kde_status kde_acc_to_real(kde_ctx *ctx, const long long *acc, int Ng, double bound, const unsigned int *wmax_bits,
                           double wscale, T *out)
{
    acc_to_real_kernel<T><<<(Ng + 255) / 256, 256, 0, ctx->stream>>>(acc, Ng, bound, wmax_bits, wscale, out);
    KDE_LAUNCHED(ctx, "acc_to_real_kernel");
    return KDE_OK;
}

template kde_status kde_deposit_sorted<float>(kde_ctx *, const uint32_t *, const float *, float, const float *, float,
                                              const float *, float, int64_t, int, double, long long *, double,
                                              const unsigned int *, double);
template kde_status kde_deposit_sorted<double>(kde_ctx *, const uint32_t *, const double *, double, const double *,
                                               double, const double *, double, int64_t, int, double, long long *,
                                               double, const unsigned int *, double);
template kde_status kde_acc_to_real<float>(kde_ctx *, const long long *, int, double, const unsigned int *, double,
                                           float *);
template kde_status kde_acc_to_real<double>(kde_ctx *, const long long *, int, double, const unsigned int *, double,
                                            double *);

// ---------------------------------------------------------------------------
// CV integral term: the deposit of every candidate on its own power-of-two
// grid of M_c points (theta units, w = 1/N), one grid per blockIdx.y.
// ---------------------------------------------------------------------------
__host__ __device__ inline int cv_grid_points(double kappa_max)
{
    // the trapezoid rule on M points integrates fhat^2 exactly up to aliased
    // modes near M/2, whose weight A_{M/2}^2 ~ exp(-(M/2)^2 / kappa) is below
    // 1e-17 once M >= 12.5 sqrt(kappa)
    double need = 12.5 * sqrt(kappa_max) + 1.0;
    int M = 64;
    while (M < need && M < CV_MAXM) M <<= 1;
    return M;
}

// per-candidate parameters of the grid deposit
struct GridPar {
    float k;       // the candidate: uniform width, or the scale of the relative widths
    float norm_u;  // uniform norm (uniform widths)
    int M;         // grid points
    int es;        // fixed-point scale 2^es of the grid sums
    float w_u;     // the weight 1/N
};

// one thread per candidate: the FP64 Bessel norm of the largest width, the grid size and
// the fixed-point scale, worked out once instead of in every thread of the deposit
__global__ void cv_grid_par_kernel(CandList cl, const unsigned int *krmax_bits, int64_t N, GridPar *par)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cl.n) return;
    const double kmax = cl.scale_mode ? cl.k[c] * (double)__uint_as_float(*krmax_bits) : cl.k[c];
    const double nb = kde_norm(kmax);  // bound of a node value: N * (1/N) * the largest norm
    GridPar p;
    p.k = (float)cl.k[c];
    p.norm_u = (float)nb;
    p.M = cv_grid_points(kmax);
    p.es = acc_scale_exp(nb);
    p.w_u = (float)(1.0 / (double)N);
    par[c] = p;
}

__global__ void __launch_bounds__(DEP_THREADS)
    cv_grid_deposit_kernel(const uint32_t *u, int64_t N, const float *kappa_rel, const float *lnorm, int scale_mode,
                           const GridPar *par, long long *acc, unsigned int *status)
{
    __shared__ float4 rsc[DEP_CHUNK];
    __shared__ float2 rwn[DEP_CHUNK];
    __shared__ float part[DEP_WARPS * DEP2_PART];
    __shared__ int red[2 * DEP_WARPS];
    const int c = blockIdx.y;
    const GridPar p = par[c];
    DepSrc<float> S{};
    S.u = u;
    S.N = N;
    S.coef = 1.0f;
    S.w = nullptr;
    S.w_u = p.w_u;
    S.nodes = nullptr;
    S.acc = acc + (size_t)c * CV_MAXM;
    S.status = status;
    S.wmax_bits = nullptr;
    S.norm = nullptr;
    if (scale_mode) {
        S.kappa = kappa_rel;
        S.kscale = p.k;
        S.lnorm = lnorm + (size_t)c * N;
    } else {
        S.kappa = nullptr;
        S.kappa_u = p.k;
        S.kscale = 1.0f;
        S.lnorm = nullptr;
        S.norm_u = p.norm_u;
    }
    S.scale_exp = p.es;
    S.Ng = p.M;
    // the CV integral term keeps the half-angle form: its sums carry the CV's accuracy
    deposit_chunk_body_x2(S, blockIdx.x, rsc, rwn, part, red, false);
}

// FP64 trapezoid sum of fhat^2 on each candidate's grid: f2[c] = (2 pi / M) sum_g fhat_g^2
__global__ void cv_grid_square_kernel(const long long *acc, const GridPar *par, double *f2)
{
    const int c = blockIdx.x;
    const int M = par[c].M;
    const double inv = __longlong_as_double((long long)(1023 - par[c].es) << 52);  // 2^-es
    __shared__ double red[256];
    double s = 0.0;
    for (int g = threadIdx.x; g < M; g += blockDim.x) {
        double f = (double)acc[(size_t)c * CV_MAXM + g] * inv;
        s += f * f;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) f2[c] = KDE_TWO_PI / M * red[0];
}

kde_status kde_cv_integral_term(kde_ctx *ctx, const uint32_t *u_sorted, int64_t N, const float *kappa_rel,
                                const float *lnorm, const unsigned int *krmax_bits, const CandList &cl,
                                double *f2_out)
{
    long long *acc = (long long *)kde_ws(ctx, WS_CV_ACC, (size_t)cl.n * CV_MAXM * sizeof(long long));
    if (!acc) return KDE_ENOMEM;
    KDE_CUDA(ctx, cudaMemsetAsync(acc, 0, (size_t)cl.n * CV_MAXM * sizeof(long long), ctx->stream), "cv acc memset");
    GridPar *par = (GridPar *)kde_ws(ctx, WS_CV_GPAR, (size_t)cl.n * sizeof(GridPar));
    if (!par) return KDE_ENOMEM;
    cv_grid_par_kernel<<<(cl.n + 63) / 64, 64, 0, ctx->stream>>>(cl, krmax_bits, N, par);
    KDE_LAUNCHED(ctx, "cv_grid_par_kernel");
    dim3 grid((unsigned)((N + DEP_CHUNK - 1) / DEP_CHUNK), (unsigned)cl.n);
    {
        KdeProfScope _ps(ctx, PROF_CV_GRID);
        cv_grid_deposit_kernel<<<grid, DEP_THREADS, 0, ctx->stream>>>(u_sorted, N, kappa_rel, lnorm, cl.scale_mode,
                                                                        par, acc, ctx->d_status);
    }
    KDE_LAUNCHED(ctx, "cv_grid_deposit_kernel");
    cv_grid_square_kernel<<<cl.n, 256, 0, ctx->stream>>>(acc, par, f2_out);
    KDE_LAUNCHED(ctx, "cv_grid_square_kernel");
    return KDE_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
template <typename T>
static kde_status deposit_api(kde_ctx *ctx, const uint32_t *u, const T *kappa, double kappa_u, const T *weight,
                              int64_t N, int Ng, double L, T *rho_out)
{
    cudaSetDevice(ctx->device);
    long long *acc = (long long *)kde_ws(ctx, WS_ACC, (size_t)Ng * sizeof(long long));
    if (!acc) return KDE_ENOMEM;
    if (N == 0) {
        KDE_CUDA(ctx, cudaMemsetAsync(rho_out, 0, (size_t)Ng * sizeof(T), ctx->stream), "rho memset");
        return KDE_OK;
    }
    uint32_t *us = (uint32_t *)kde_ws(ctx, WS_SORT_U, (size_t)N * 4);
    T *ks = kappa ? (T *)kde_ws(ctx, WS_SORT_P0, (size_t)N * sizeof(T)) : nullptr;
    T *ws = weight ? (T *)kde_ws(ctx, WS_SORT_P1, (size_t)N * sizeof(T)) : nullptr;
    if (!us || (kappa && !ks) || (weight && !ws)) return KDE_ENOMEM;
    SortPayload pl[2];
    int npl = 0;
    if (kappa) pl[npl++] = SortPayload{kappa, ks, (int)sizeof(T)};
    if (weight) pl[npl++] = SortPayload{weight, ws, (int)sizeof(T)};
    KDE_TRY(kde_sort_by_bin(ctx, u, N, Ng, us, pl, npl, nullptr));
    const double coef = KDE_TWO_PI / L;
    double norm_u = kappa ? 0.0 : kde_norm(kappa_u);
    double norm_bound = kappa ? kde_norm(KDE_KAPPA_MAX) : norm_u;
    double w_u = L / (double)N;
    unsigned int *wmax = nullptr;
    double bound = (double)N * w_u * coef * norm_bound;
    if (weight) {
        wmax = (unsigned int *)kde_ws(ctx, WS_WMAX, 64);
        if (!wmax) return KDE_ENOMEM;
        KDE_CUDA(ctx, cudaMemsetAsync(wmax, 0, 4, ctx->stream), "wmax memset");
        int blocks = (int)((N + 255) / 256);
        blocks = blocks > ctx->sm_count * 8 ? ctx->sm_count * 8 : blocks;
        wmax_kernel<T><<<blocks, 256, 0, ctx->stream>>>(weight, N, wmax, ctx->d_status);
        KDE_LAUNCHED(ctx, "wmax_kernel");
    }
    KDE_TRY(kde_deposit_sorted<T>(ctx, us, ks, (T)kappa_u, nullptr, (T)norm_u, ws, (T)w_u, N, Ng, coef, acc, bound,
                                  wmax, norm_bound));
    return kde_acc_to_real<T>(ctx, acc, Ng, bound, wmax, (double)N * coef * norm_bound, rho_out);
}

extern "C" kde_status kde_deposit(kde_ctx *ctx, const uint32_t *u, const void *kappa, double kappa_uniform,
                                  const void *weight, int64_t N, int32_t Ng, double L, void *rho_out, uint32_t flags)
{
    if (!ctx) return KDE_EINVAL;
    if (N < 0 || Ng < 1 || Ng > KDE_MAX_NG || !(L > 0) || !rho_out || (N > 0 && !u))
        return kde_fail(ctx, KDE_EINVAL, "kde_deposit: need N >= 0, 1 <= Ng <= %d, L > 0, non-null u and rho_out",
                        KDE_MAX_NG);
    if (!kappa && !(kappa_uniform > 0 && kappa_uniform <= KDE_KAPPA_MAX))
        return kde_fail(ctx, KDE_EINVAL, "kde_deposit: kappa_uniform must be in (0, 1e6]");
    if (N > 0xFFFFFFFFll) return kde_fail(ctx, KDE_EINVAL, "kde_deposit: N must be below 2^32");
    if (flags & ~KDE_F64) return kde_fail(ctx, KDE_ENOTSUP, "kde_deposit: unsupported flags 0x%x", flags);
    if (flags & KDE_F64)
        return deposit_api<double>(ctx, u, (const double *)kappa, kappa_uniform, (const double *)weight, N, Ng, L,
                                   (double *)rho_out);
    return deposit_api<float>(ctx, u, (const float *)kappa, kappa_uniform, (const float *)weight, N, Ng, L,
                              (float *)rho_out);
}

// ---------------------------------------------------------------------------
// Allocation-free deposit.
//
// Some callers cannot call cudaMalloc once they are running: code that records
// its work into a CUDA graph or runs under a host allocator policy that
// forbids device allocations after start-up, plugins that must not touch the
// host process's memory pools, and real-time loops that may not block on the
// driver's allocator.  kde_deposit_noalloc serves them: it needs no context and
// no workspace.  Particles may come in any order (nothing is sorted); every
// scratch byte it uses -- the int64 grid accumulators, the node table and the
// largest-weight word -- lives in the file-scope array below, which every GPU
// that loads this library holds (KDE_NOALLOC_SCRATCH_BYTES) until the process
// exits.  Every call shares that one array: calls that overlap on the GPU
// (concurrent streams, or several host threads) race on it.
// ---------------------------------------------------------------------------
#define NOALLOC_ACC_OFF 0
#define NOALLOC_NODE_OFF (KDE_MAX_NG * 8)
#define NOALLOC_WMAX_OFF (NOALLOC_NODE_OFF + KDE_MAX_NG * 16)
static_assert(KDE_NOALLOC_SCRATCH_BYTES >= NOALLOC_WMAX_OFF + 256, "scratch layout exceeds the declared size");

static __device__ __align__(256) unsigned char kde_noalloc_scratch[KDE_NOALLOC_SCRATCH_BYTES];

template <typename T>
__global__ void __launch_bounds__(DEP_THREADS) deposit_chunk_unsorted_kernel(DepSrc<T> S)
{
    __shared__ DepRec<T> rec[DEP_CHUNK];
    __shared__ T part[DEP_WARPS * 32 * DEP_WARPS];
    __shared__ int red[DEP_WARPS];
    __shared__ int cmm[2 * DEP_WARPS];
    deposit_chunk_body<T, true>(S, blockIdx.x, rec, part, red, cmm);
}

template <typename T2>
__global__ void noalloc_node_kernel(T2 *tab, int Ng)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Ng) return;
    double s, c;
    sincospi((double)g / (double)Ng, &s, &c);
    tab[g].x = s;
    tab[g].y = c;
}

// device address of the scratch array on the current device.  Looked up on every
// call (a host-side table lookup once the module is loaded): a cached address
// would go stale if the device's context were reset and the module reloaded.
static unsigned char *noalloc_scratch_address()
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, kde_noalloc_scratch) != cudaSuccess || !p) return nullptr;
    return (unsigned char *)p;
}

// every launch goes through cudaLaunchKernel, whose return value is that launch's
// own status (a trailing cudaGetLastError would also report, and clear, errors of
// unrelated earlier launches on this thread)
template <typename T>
static kde_status deposit_noalloc_impl(cudaStream_t stream, unsigned char *scr, const uint32_t *u, const T *kappa,
                                       double kappa_u, const T *weight, int64_t N, int Ng, double L, T *rho_out)
{
    typedef typename V2<T>::t T2;
    long long *acc = (long long *)(scr + NOALLOC_ACC_OFF);
    T2 *nodes = (T2 *)(scr + NOALLOC_NODE_OFF);
    unsigned int *wmax = (unsigned int *)(scr + NOALLOC_WMAX_OFF);
    if (cudaMemsetAsync(acc, 0, (size_t)Ng * sizeof(long long), stream) != cudaSuccess) return KDE_ECUDA;
    if (N == 0) return cudaMemsetAsync(rho_out, 0, (size_t)Ng * sizeof(T), stream) == cudaSuccess ? KDE_OK : KDE_ECUDA;
    {
        void *args[] = {&nodes, &Ng};
        if (cudaLaunchKernel((const void *)noalloc_node_kernel<T2>, dim3((Ng + 255) / 256), dim3(256), args, 0,
                             stream) != cudaSuccess)
            return KDE_ECUDA;
    }
    const double coef = KDE_TWO_PI / L;
    const double norm_u = kappa ? 0.0 : kde_norm(kappa_u);
    const double norm_bound = kappa ? kde_norm(KDE_KAPPA_MAX) : norm_u;
    const double w_u = L / (double)N;
    double bound = (double)N * w_u * coef * norm_bound;
    if (weight) {
        if (cudaMemsetAsync(wmax, 0, 4, stream) != cudaSuccess) return KDE_ECUDA;
        int blocks = (int)((N + 255) / 256);
        blocks = blocks > 1024 ? 1024 : blocks;
        unsigned int *no_status = nullptr;
        void *args[] = {(void *)&weight, &N, &wmax, &no_status};
        if (cudaLaunchKernel((const void *)wmax_kernel<T>, dim3(blocks), dim3(256), args, 0, stream) != cudaSuccess)
            return KDE_ECUDA;
    }
    DepSrc<T> S{};
    S.u = u;
    S.N = N;
    S.kappa = kappa;
    S.kappa_u = (T)kappa_u;
    S.kscale = (T)1;
    S.norm_u = (T)norm_u;
    S.w = weight;
    S.w_u = (T)w_u;
    S.coef = (T)coef;
    S.Ng = Ng;
    S.nodes = nodes;
    S.acc = acc;
    S.bound = bound;
    S.wmax_bits = weight ? wmax : nullptr;
    S.norm_bound = norm_bound;
    S.status = nullptr;
    {
        void *args[] = {&S};
        if (cudaLaunchKernel((const void *)deposit_chunk_unsorted_kernel<T>,
                             dim3((unsigned)((N + DEP_CHUNK - 1) / DEP_CHUNK)), dim3(DEP_THREADS), args, 0,
                             stream) != cudaSuccess)
            return KDE_ECUDA;
    }
    {
        const unsigned int *wb = weight ? wmax : nullptr;
        double wscale = (double)N * coef * norm_bound;
        void *args[] = {&acc, &Ng, &bound, (void *)&wb, &wscale, &rho_out};
        if (cudaLaunchKernel((const void *)acc_to_real_kernel<T>, dim3((Ng + 255) / 256), dim3(256), args, 0,
                             stream) != cudaSuccess)
            return KDE_ECUDA;
    }
    return KDE_OK;
}

extern "C" kde_status kde_deposit_noalloc(void *stream, const uint32_t *u, const void *kappa, double kappa_uniform,
                                          const void *weight, int64_t N, int32_t Ng, double L, void *rho_out,
                                          uint32_t flags)
{
    if (N < 0 || N > 0xFFFFFFFFll || Ng < 1 || Ng > KDE_NOALLOC_MAX_NG || !(L > 0) || !rho_out || (N > 0 && !u))
        return KDE_EINVAL;
    if (!kappa && !(kappa_uniform > 0 && kappa_uniform <= KDE_KAPPA_MAX)) return KDE_EINVAL;
    if (flags & ~KDE_F64) return KDE_ENOTSUP;
    unsigned char *scr = noalloc_scratch_address();
    if (!scr) return KDE_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    if (flags & KDE_F64)
        return deposit_noalloc_impl<double>(s, scr, u, (const double *)kappa, kappa_uniform, (const double *)weight, N,
                                            Ng, L, (double *)rho_out);
    return deposit_noalloc_impl<float>(s, scr, u, (const float *)kappa, kappa_uniform, (const float *)weight, N, Ng, L,
                                       (float *)rho_out);
}
