// cv.cu -- leave-one-out cross-validation over candidate widths (Sec. II.B,
// Eq. cv_def) and Silverman's particle-wise widths (Sec. II.C).
//
// CV_theta(c) = int fhat_c^2 dtheta - 2/(n(n-1)) sum_i sum_{j != i} K_{kappa_jc}(theta_i - theta_j)
//
// Pair term.  Particles are bin-sorted and cut into tiles of CV_T = 256.  A CTA
// owns one "row" tile (one particle per thread, kept in registers) and walks
// "column" tiles outward from its own; each column tile's half-angle (sin,
// cos) pairs are staged into shared memory with a 1D TMA bulk copy
// (cp.async.bulk + mbarrier, double-buffered).  For a pair the kernel forms
// s = sin((theta_j - theta_i)/2) by the angle-difference identity (2 FMA-pipe
// ops), s^2 once, and then for every active candidate one FMUL/FFMA, one
// ex2.approx and one FADD.  Candidates are sorted by width; a tile pair whose
// angular gap exceeds a candidate's truncation radius (kernel < 2^-24 of its
// peak) skips that candidate, and the walk stops when no candidate reaches.
// Uniform widths are symmetric, so only unordered tile pairs are visited
// (weight 2 off the diagonal); per-particle widths visit ordered pairs.
// Per-thread FP32 sums of one tile are reduced across the warp and added to
// FP64 accumulators; per-CTA partials are reduced in a fixed order, so the
// result is deterministic.
//
// Integral term: exact trapezoid sum of fhat^2 on a power-of-two grid fine
// enough for each candidate (deposit.cu).  Combination and argmin in FP64.
#include "common.cuh"

#define CV_T 256
#define CV_WARPS (CV_T / 32)
#define CV_G 8
#define CV_MAXC 256
#define CV_WAIT_LIMIT (1u << 26)

// internal candidate order (ascending width) plus the map back to the caller's order
struct CvCands {
    int n;
    int scale_mode;
    float k[CV_MAXC];      // sorted candidate widths (uniform) or scale factors
    int orig[CV_MAXC];     // sorted position -> caller index
};

kde_status kde_cv_integral_term(kde_ctx *ctx, const uint32_t *u_sorted, int64_t N, const float *kappa_rel,
                                const float *lnorm, const unsigned int *krmax_bits, const CandList &cl,
                                double *f2_out);

// ---------------------------------------------------------------------------
// TMA / mbarrier helpers (bounded waits)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// returns false if the phase did not complete within `limit` polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned limit = CV_WAIT_LIMIT)
{
    for (unsigned it = 0; it < limit; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Wait for the staged tile of buffer `cur`.  Thread 0 polls with the context's
// limit (`polls`) and broadcasts the outcome; on success every other thread
// observes the completed phase too (its wait returns at once), so all of them
// read the tile after the barrier's acquire.  On failure every copy still in
// flight -- the late one and the prefetch issued after it -- is waited for with
// the full limit before the caller leaves, so no bulk copy lands in shared
// memory that the CTA has given up.  Returns false on failure (the caller flags
// KDE_DEV_WAIT_TIMEOUT and stops).
__device__ __forceinline__ bool tile_wait(uint64_t *bar, unsigned *phase, int cur, bool next_pending, unsigned polls,
                                          int *s_stop, unsigned int *status)
{
    const int tid = threadIdx.x;
    if (tid == 0) *s_stop = mbar_wait(&bar[cur], phase[cur], polls) ? 0 : 1;
    __syncthreads();
    if (*s_stop) {
        const bool a = mbar_wait(&bar[cur], phase[cur]);
        const bool b = !next_pending || mbar_wait(&bar[cur ^ 1], phase[cur ^ 1]);
        if (tid == 0 && !(a && b)) kde_flag(status, KDE_DEV_WAIT_TIMEOUT, 0xffffffffu);
        return false;
    }
    if (tid != 0) mbar_wait(&bar[cur], phase[cur]);
    phase[cur] ^= 1u;
    return true;
}

// ---------------------------------------------------------------------------
// geometry helpers
// ---------------------------------------------------------------------------
// circular gap (in position-code units) between the code intervals of two tiles
__device__ __forceinline__ uint32_t tile_gap(uint2 a, uint2 b)
{
    if ((uint32_t)(b.x - a.x) <= (uint32_t)(a.y - a.x)) return 0u;  // b starts inside a
    if ((uint32_t)(a.x - b.x) <= (uint32_t)(b.y - b.x)) return 0u;  // a starts inside b
    uint32_t g1 = b.x - a.y, g2 = a.x - b.y;
    return g1 < g2 ? g1 : g2;
}
// largest width whose truncated kernel still reaches across a gap
__device__ __forceinline__ float reach_kappa(uint32_t gap)
{
    if (gap == 0u) return 3.0e38f;
    float s = sinpif((float)gap * (1.0f / 4294967296.0f));  // sin(gap_theta / 2)
    return (float)(KDE_XCUT * KDE_LN2 / 2.0) / (s * s);
}

// ---------------------------------------------------------------------------
// prep: per-particle half-angle (sin, cos); per-tile code interval, widened to
// whole sort bins so that tile intervals are monotone along the sorted order;
// for per-particle widths also the exponent factor, the tile's smallest width,
// the global extremes and log2 of every (particle, candidate) normalisation
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(CV_T)
    cv_prep_kernel(const uint32_t *u, const float *kr, int64_t N, int bin_shift, float2 *sc, uint2 *tile_u,
                   float *tile_kmin, float *k2rel, unsigned int *kr_bits, CandList cl, float *lnorm,
                   unsigned int *status, const float2 *ntab)
{
    __shared__ float skmin[CV_WARPS];
    const int64_t j = (int64_t)blockIdx.x * CV_T + threadIdx.x;
    const bool valid = j < N;
    uint32_t uu = valid ? u[j] : 0u;
    float s = 0.f, c = 1.f;
    if (valid) kde_half_sincos(uu, s, c);
    sc[j] = make_float2(s, c);
    if (threadIdx.x == 0) {
        int64_t last = (int64_t)blockIdx.x * CV_T + CV_T - 1;
        if (last >= N) last = N - 1;
        uint32_t b0 = u[(int64_t)blockIdx.x * CV_T] >> bin_shift, b1 = u[last] >> bin_shift;
        tile_u[blockIdx.x] = make_uint2(b0 << bin_shift, ((b1 + 1u) << bin_shift) - 1u);
    }
    if (kr) {
        float k = valid ? kr[j] : 1.0f;
        if (valid && !(k > 0.f && k <= (float)KDE_KAPPA_MAX)) {
            kde_flag(status, KDE_DEV_KAPPA_RANGE, (unsigned)j);
            k = 1.0f;
        }
        k2rel[j] = (float)(-2.0 * KDE_LOG2E) * k;
        float km = valid ? k : 3.0e38f;
        if (valid) {
            atomicMax(&kr_bits[0], __float_as_uint(k));
            atomicMin(&kr_bits[1], __float_as_uint(k));
            // log2 of the tabulated FP32 norm (FP64 Bessel series per particle and candidate are slow here)
            for (int q = 0; q < cl.n; ++q)
                lnorm[(size_t)q * N + j] = log2f(kde_norm_tab(ntab, (float)(cl.k[q] * (double)k)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) km = fminf(km, __shfl_xor_sync(0xffffffffu, km, o));
        if ((threadIdx.x & 31) == 0) skmin[threadIdx.x >> 5] = km;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < CV_WARPS; ++w) km = fminf(km, skmin[w]);
            tile_kmin[blockIdx.x] = fminf(km, skmin[0]);
        }
    }
}

// ---------------------------------------------------------------------------
// tile walk: from row tile a, the column tiles whose gap a kernel of width
// Kthr can bridge form (at most) a forward run a, a+1, ... and a backward run
// a-1, a-2, ... (tile intervals are monotone, so the forward and backward gaps
// are monotone in the step).  The walk visits both runs once each.
// ---------------------------------------------------------------------------
struct Walk {
    int phase, k, F;
};

__device__ __forceinline__ bool walk_next(Walk &w, int a, int NT, const uint2 *tile_u, uint2 ta, float Kthr, int &b,
                                          int &d)
{
    for (;;) {
        if (w.phase == 0) {
            if (w.k >= NT) {
                w.phase = 2;
                return false;
            }
            int bb = (a + w.k) % NT;
            if (w.k == 0 || Kthr <= reach_kappa(tile_gap(ta, tile_u[bb]))) {
                b = bb;
                d = w.k;
                w.F = w.k;
                ++w.k;
                return true;
            }
            w.phase = 1;
            w.k = 1;
        } else if (w.phase == 1) {
            if (w.k >= NT - w.F) {
                w.phase = 2;
                return false;
            }
            int bb = ((a - w.k) % NT + NT) % NT;
            if (Kthr <= reach_kappa(tile_gap(ta, tile_u[bb]))) {
                b = bb;
                d = -w.k;
                ++w.k;
                return true;
            }
            w.phase = 2;
            return false;
        } else {
            return false;
        }
    }
}

// unordered tile pairs are visited from the tile with the smaller forward
// offset: d = (b - a) mod NT <= NT/2, and for even NT the half-way pair only
// from the first half
__device__ __forceinline__ bool canonical_pair(int a, int b, int NT)
{
    int d = ((b - a) % NT + NT) % NT;
    if (2 * d < NT) return true;
    if (2 * d == NT) return a < NT / 2;
    return false;
}

// ---------------------------------------------------------------------------
// pair totals over all active candidates
// ---------------------------------------------------------------------------
struct CvPairArgs {
    const float2 *sc;
    int64_t N;
    int NT;
    int splits;
    const uint2 *tile_u;
    const float *tile_kmin;  // per-particle widths only
    const float *k2rel;
    const float *lnorm;
    double *part;  // [gridDim.x][n]
    unsigned int *status;
    unsigned wait_polls;  // polls of a tile wait before the kernel gives up
};

template <bool SCALE>
__device__ __forceinline__ int active_candidates(const CvCands &cc, uint32_t gap, float kmin)
{
    float kr = reach_kappa(gap);
    int c = 0;
    if (SCALE) {
        while (c < cc.n && cc.k[c] * kmin <= kr) ++c;
    } else {
        while (c < cc.n && cc.k[c] <= kr) ++c;
    }
    return c;
}

template <bool SCALE>
__global__ void __launch_bounds__(CV_T) cv_pairs_kernel(CvPairArgs A, CvCands cc)
{
    __shared__ __align__(128) float2 buf[2][CV_T];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ double wacc[CV_WARPS][CV_MAXC];
    __shared__ int s_stop;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int a = blockIdx.x / A.splits, sidx = blockIdx.x % A.splits;
    const int NT = A.NT;
    for (int c = tid; c < CV_WARPS * CV_MAXC; c += CV_T) (&wacc[0][0])[c] = 0.0;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_barrier_init();
    }
    const int64_t j = (int64_t)a * CV_T + tid;
    const bool rvalid = j < A.N;
    const float2 me = A.sc[j];
    const float rmask = rvalid ? 1.0f : 0.0f;
    const float k2r = SCALE ? (rvalid ? A.k2rel[j] : 0.f) : 0.f;
    const uint2 ta = A.tile_u[a];
    const float kmin_a = SCALE ? A.tile_kmin[a] : 1.0f;
    const float Kthr = cc.k[0] * kmin_a;  // the widest kernel of this row tile
    __syncthreads();

    Walk w{0, 0, 0};
    int cnt = 0;
    // next column tile assigned to this CTA (every CTA of the row walks the same sequence)
    auto fetch = [&](int &b, int &d) -> bool {
        while (walk_next(w, a, NT, A.tile_u, ta, Kthr, b, d)) {
            if (!SCALE && !canonical_pair(a, b, NT)) continue;
            if ((cnt++) % A.splits == sidx) return true;
        }
        return false;
    };
    int b_cur = 0, d_cur = 0;
    bool have = fetch(b_cur, d_cur);
    if (have && tid == 0) tma_load_1d(buf[0], A.sc + (size_t)b_cur * CV_T, CV_T * sizeof(float2), &bar[0]);
    unsigned phase[2] = {0u, 0u};
    bool failed = false;
    for (int k = 0; have; ++k) {
        const int cur = k & 1;
        int b_nxt = 0, d_nxt = 0;
        const bool next = fetch(b_nxt, d_nxt);
        if (next && tid == 0)
            tma_load_1d(buf[cur ^ 1], A.sc + (size_t)b_nxt * CV_T, CV_T * sizeof(float2), &bar[cur ^ 1]);
        if (!tile_wait(bar, phase, cur, next, A.wait_polls, &s_stop, A.status)) {
            failed = true;
            break;
        }
        const int b = b_cur;
        const int nact = active_candidates<SCALE>(cc, tile_gap(ta, A.tile_u[b]), kmin_a);
        if (nact > 0) {
            const int64_t col0 = (int64_t)b * CV_T;
            const int ncol = (int)(A.N - col0 < CV_T ? A.N - col0 : CV_T);
            const bool diag = (d_cur == 0);
            const float wgt = (!SCALE && !diag) ? 2.0f : 1.0f;
            const float2 *t = buf[cur];
            for (int cg = 0; cg < nact; cg += CV_G) {
                // candidates in packed pairs: exponent s^2 kk + ll, two exp2, one add per pair
                float kk[CV_G], ll[CV_G], acc[CV_G];
#pragma unroll
                for (int q = 0; q < CV_G; ++q) {
                    int c = cg + q < nact ? cg + q : nact - 1;
                    if (SCALE) {
                        kk[q] = cc.k[c] * k2r;
                        ll[q] = rvalid ? A.lnorm[(size_t)c * A.N + j] : 0.f;
                    } else {
                        kk[q] = (float)(-2.0 * KDE_LOG2E) * cc.k[c];
                        ll[q] = 0.f;
                    }
                }
                kde_f2 kk2[CV_G / 2], ll2[CV_G / 2], acc2[CV_G / 2];
#pragma unroll
                for (int p = 0; p < CV_G / 2; ++p) {
                    kk2[p] = kde_pk(kk[2 * p], kk[2 * p + 1]);
                    ll2[p] = kde_pk(ll[2 * p], ll[2 * p + 1]);
                    acc2[p] = kde_pk(0.f, 0.f);
                }
                const kde_f2 one2 = kde_pk(1.f, 1.f);
                auto column = [&](int i) {
                    const float2 o = t[i];
                    const float s = me.x * o.y - me.y * o.x;
                    const float s2 = s * s;
                    const kde_f2 s22 = kde_pk(s2, s2);
#pragma unroll
                    for (int p = 0; p < CV_G / 2; ++p)
                        acc2[p] = kde_fma2(kde_ex22(kde_fma2(s22, kk2[p], ll2[p])), one2, acc2[p]);
                };
                if (!diag) {
#pragma unroll 2
                    for (int i = 0; i < ncol; ++i) column(i);
                } else {
                    for (int i = 0; i < ncol; ++i)
                        if (i != tid) column(i);
                }
#pragma unroll
                for (int p = 0; p < CV_G / 2; ++p) kde_upk(acc2[p], acc[2 * p], acc[2 * p + 1]);
#pragma unroll
                for (int q = 0; q < CV_G; ++q) {
                    float v = acc[q] * rmask;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0 && cg + q < nact) wacc[warp][cg + q] += (double)wgt * (double)v;
                }
            }
        }
        __syncthreads();  // buffer `cur` is free again
        b_cur = b_nxt;
        d_cur = d_nxt;
        have = next;
    }
    if (failed && tid == 0) kde_flag(A.status, KDE_DEV_WAIT_TIMEOUT, (unsigned)blockIdx.x);
    __syncthreads();
    for (int c = tid; c < cc.n; c += CV_T) {
        double s = 0.0;
        for (int ww = 0; ww < CV_WARPS; ++ww) s += wacc[ww][c];
        A.part[(size_t)blockIdx.x * cc.n + c] = s;
    }
}

// ---------------------------------------------------------------------------
// Uniform widths, at most 64 candidates: persistent pair kernel.
//
// Work items are (row tile, split) pairs handed out by an atomic counter; each
// item's FP64 sums go to the item's own slot, so the result does not depend on
// which CTA ran which item.  Per column particle the kernel forms s^2 once and
// then runs every active candidate with its exponent factor -2 kappa_c log2 e
// read as a constant-bank operand.  The number of active candidates of a tile
// pair, rounded up to a multiple of 4, selects one of 16 instantiations of the
// column loop, so no per-column branching remains.  After each tile pair the
// 64 per-thread FP32 sums are reduced across the warp by a transposing
// butterfly (62 shuffles leave lane l with candidates l and l + 32), and added
// to per-warp FP64 accumulators.
// ---------------------------------------------------------------------------
#define CVF_MAXC 64

struct CvFast {
    int n;             // active candidates (sorted ascending by width)
    int nitems;        // work items = row tiles x splits
    int splits;
    float kk[CVF_MAXC];  // -2 log2(e) kappa_c
    float k[CVF_MAXC];   // kappa_c
    kde_f2 kk2[CVF_MAXC / 2];  // (kk[2p], kk[2p + 1]) as packed pairs
};

// candidates in packed pairs: per column one exponent s^2, then for each pair of
// candidates one f32x2 multiply, two exp2 and one f32x2 add (as a multiply-add by 1)
template <int NG>
__device__ __forceinline__ void cvf_columns(const float2 *__restrict__ t, int ncol, float2 me, int self,
                                            kde_f2 (&acc)[CVF_MAXC / 2], const CvFast &cf)
{
    const kde_f2 one2 = kde_pk(1.f, 1.f);
    auto column = [&](int i) {
        const float2 o = t[i];
        const float s = me.x * o.y - me.y * o.x;
        const float s2 = s * s;
        const kde_f2 s22 = kde_pk(s2, s2);
#pragma unroll
        for (int p = 0; p < 2 * NG; ++p) acc[p] = kde_fma2(kde_ex22(kde_mul2(s22, cf.kk2[p])), one2, acc[p]);
    };
    if (self < 0) {
#pragma unroll 2
        for (int i = 0; i < ncol; ++i) column(i);
    } else {
        for (int i = 0; i < ncol; ++i)
            if (i != self) column(i);
    }
}

__device__ __forceinline__ void cvf_dispatch(int ng, const float2 *t, int ncol, float2 me, int self,
                                             kde_f2 (&acc)[CVF_MAXC / 2], const CvFast &cf)
{
    switch (ng) {
#define CVF_CASE(G) \
    case G: cvf_columns<G>(t, ncol, me, self, acc, cf); break;
        CVF_CASE(1) CVF_CASE(2) CVF_CASE(3) CVF_CASE(4) CVF_CASE(5) CVF_CASE(6) CVF_CASE(7) CVF_CASE(8)
        CVF_CASE(9) CVF_CASE(10) CVF_CASE(11) CVF_CASE(12) CVF_CASE(13) CVF_CASE(14) CVF_CASE(15) CVF_CASE(16)
#undef CVF_CASE
    default: break;
    }
}

// butterfly over 32 values: afterwards lane l holds the warp sum of v[l]
__device__ __forceinline__ float warp_transpose_sum32(float (&v)[32], int lane)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            float send = up ? v[i] : v[i + o];
            float keep = up ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

__global__ void __launch_bounds__(CV_T, 2)
    cv_pairs_fast_kernel(const float2 *__restrict__ sc, int64_t N, int NT, const uint2 *__restrict__ tile_u,
                         int *counter, double *part, unsigned int *status, unsigned wait_polls,
                         const __grid_constant__ CvFast cf)
{
    __shared__ __align__(128) float2 buf[2][CV_T];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ double wacc[CV_WARPS][CVF_MAXC];
    __shared__ int s_item, s_stop;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_barrier_init();
    }
    unsigned phase[2] = {0u, 0u};
    bool failed = false;
    const float Kthr = cf.k[0];
    for (;;) {
        __syncthreads();  // the previous item's readers of s_item and wacc are done
        if (tid == 0) s_item = atomicAdd(counter, 1);
        for (int c = tid; c < CV_WARPS * CVF_MAXC; c += CV_T) (&wacc[0][0])[c] = 0.0;
        __syncthreads();
        const int item = s_item;
        if (item >= cf.nitems) break;
        const int a = item / cf.splits, sidx = item % cf.splits;
        const int64_t j = (int64_t)a * CV_T + tid;
        const bool rvalid = j < N;
        const float2 me = sc[j];
        const uint2 ta = tile_u[a];
        kde_f2 acc[CVF_MAXC / 2];
#pragma unroll
        for (int p = 0; p < CVF_MAXC / 2; ++p) acc[p] = kde_pk(0.f, 0.f);

        Walk w{0, 0, 0};
        int cnt = 0;
        auto fetch = [&](int &b, int &d) -> bool {
            while (walk_next(w, a, NT, tile_u, ta, Kthr, b, d)) {
                if (!canonical_pair(a, b, NT)) continue;
                if ((cnt++) % cf.splits == sidx) return true;
            }
            return false;
        };
        int b_cur = 0, d_cur = 0;
        bool have = fetch(b_cur, d_cur);
        int cur = 0;
        if (have && tid == 0) tma_load_1d(buf[cur], sc + (size_t)b_cur * CV_T, CV_T * sizeof(float2), &bar[cur]);
        while (have) {
            int b_nxt = 0, d_nxt = 0;
            const bool next = fetch(b_nxt, d_nxt);
            if (next && tid == 0)
                tma_load_1d(buf[cur ^ 1], sc + (size_t)b_nxt * CV_T, CV_T * sizeof(float2), &bar[cur ^ 1]);
            if (!tile_wait(bar, phase, cur, next, wait_polls, &s_stop, status)) {
                failed = true;
                break;
            }
            // active candidates of this tile pair (widths sorted ascending)
            const float kr = reach_kappa(tile_gap(ta, tile_u[b_cur]));
            int nact = 0;
            while (nact < cf.n && cf.k[nact] <= kr) ++nact;
            if (nact > 0) {
                const int64_t col0 = (int64_t)b_cur * CV_T;
                const int ncol = (int)(N - col0 < CV_T ? N - col0 : CV_T);
                const bool diag = d_cur == 0;
                cvf_dispatch((nact + 3) >> 2, buf[cur], ncol, me, diag ? tid : -1, acc, cf);
                const float wgt = diag ? 1.0f : 2.0f;
                const float m = rvalid ? wgt : 0.0f;
                float lo[32], hi[32];
#pragma unroll
                for (int p = 0; p < 16; ++p) {
                    float a0, a1, b0, b1;
                    kde_upk(acc[p], a0, a1);
                    kde_upk(acc[p + 16], b0, b1);
                    lo[2 * p] = a0 * m;
                    lo[2 * p + 1] = a1 * m;
                    hi[2 * p] = b0 * m;
                    hi[2 * p + 1] = b1 * m;
                    acc[p] = kde_pk(0.f, 0.f);
                    acc[p + 16] = kde_pk(0.f, 0.f);
                }
                const float r0 = warp_transpose_sum32(lo, lane);
                const float r1 = warp_transpose_sum32(hi, lane);
                wacc[warp][lane] += (double)r0;
                wacc[warp][lane + 32] += (double)r1;
            }
            __syncthreads();  // buffer `cur` is free again
            cur ^= 1;
            b_cur = b_nxt;
            d_cur = d_nxt;
            have = next;
        }
        if (failed) {
            if (tid == 0) kde_flag(status, KDE_DEV_WAIT_TIMEOUT, (unsigned)blockIdx.x);
            break;
        }
        __syncthreads();
        for (int c = tid; c < cf.n; c += CV_T) {
            double sum = 0.0;
            for (int ww = 0; ww < CV_WARPS; ++ww) sum += wacc[ww][c];
            part[(size_t)item * cf.n + c] = sum;
        }
    }
}

// per-candidate sum of CTA partials in CTA order
__global__ void cv_reduce_kernel(const double *part, int nblocks, int n, double *tot)
{
    const int c = blockIdx.x;
    __shared__ double red[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 256) s += part[(size_t)b * n + c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) tot[c] = red[0];
}

// CV in x units for every candidate (caller's order), argmin (smallest caller
// index on exact ties) and the selected width
__global__ void cv_combine_kernel(const double *f2, const double *tot, CvCands cc, CandList cl, int64_t N,
                                  double L, double *cv_out, int *argmin, double *kstar)
{
    if (threadIdx.x != 0) return;
    const double n = (double)N, xs = KDE_TWO_PI / L;
    for (int c = 0; c < cc.n; ++c) {
        double t = tot[c];
        if (!cc.scale_mode) t *= kde_norm((double)cl.k[c]);
        cv_out[cc.orig[c]] = xs * (f2[c] - 2.0 * t / (n * (n - 1.0)));
    }
    int best = 0;
    for (int c = 1; c < cc.n; ++c)
        if (cv_out[c] < cv_out[best]) best = c;
    *argmin = best;
    if (kstar) {
        // the caller-order candidate value
        for (int c = 0; c < cc.n; ++c)
            if (cc.orig[c] == best) *kstar = cl.k[c];
    }
}

// ---------------------------------------------------------------------------
// leave-one-out sums at the selected candidate (rows = targets, columns =
// sources with their own kernels), written in the caller's particle order
// ---------------------------------------------------------------------------
struct CvLooArgs {
    const float2 *sc;
    int64_t N;
    int NT;
    const uint2 *tile_u;
    const float *tile_kmin;
    const float *k2rel;
    const float *lnorm;
    const uint32_t *perm;
    const int *argmin;  // caller index
    const unsigned int *kr_bits;  // [0] largest, [1] smallest per-particle width (float bits)
    CvCands cc;
    double xs;  // 2 pi / L
    float *loo;
};

template <bool SCALE>
__global__ void __launch_bounds__(CV_T) cv_loo_kernel(CvLooArgs A)
{
    __shared__ float2 tsc[CV_T];
    __shared__ float2 tkl[CV_T];
    const int tid = threadIdx.x;
    const int a = blockIdx.x, NT = A.NT;
    // sorted position of the selected candidate
    const int best = *A.argmin;
    int cs = 0;
    for (int c = 0; c < A.cc.n; ++c)
        if (A.cc.orig[c] == best) cs = c;
    const float kc = A.cc.k[cs];
    const int64_t i = (int64_t)a * CV_T + tid;
    const bool rvalid = i < A.N;
    const float2 me = A.sc[i];
    const uint2 ta = A.tile_u[a];
    // sources carry their own widths: walk with the smallest width anywhere (a bound)
    const float Kthr = SCALE ? kc * __uint_as_float(A.kr_bits[1]) : kc;
    const float kk = (float)(-2.0 * KDE_LOG2E) * kc;
    double sum = 0.0;
    Walk w{0, 0, 0};
    int b, d;
    while (walk_next(w, a, NT, A.tile_u, ta, Kthr, b, d)) {
        if (SCALE && !(kc * A.tile_kmin[b] <= reach_kappa(tile_gap(ta, A.tile_u[b])))) continue;
        const int64_t j = (int64_t)b * CV_T + tid;
        __syncthreads();
        tsc[tid] = A.sc[j];
        if (SCALE) {
            float k2 = j < A.N ? A.k2rel[j] * kc : 0.f;
            float l = j < A.N ? A.lnorm[(size_t)cs * A.N + j] : 0.f;
            tkl[tid] = make_float2(k2, l);
        }
        __syncthreads();
        const int ncol = (int)(A.N - (int64_t)b * CV_T < CV_T ? A.N - (int64_t)b * CV_T : CV_T);
        float acc = 0.f;
        for (int q = 0; q < ncol; ++q) {
            if (d == 0 && q == tid) continue;
            float2 o = tsc[q];
            float s = me.x * o.y - me.y * o.x;
            float s2 = s * s;
            if (SCALE) {
                float2 p = tkl[q];
                acc += kde_ex2(fmaf(s2, p.x, p.y));
            } else {
                acc += kde_ex2(s2 * kk);
            }
        }
        sum += (double)acc;
    }
    if (!rvalid) return;
    if (!SCALE) sum *= kde_norm((double)kc);
    const double loo = A.xs * sum / (double)(A.N - 1);
    A.loo[A.perm ? A.perm[i] : i] = (float)loo;
}

// ---------------------------------------------------------------------------
// Leave-one-out sums at the selected width, uniform widths: one row tile per
// CTA, column tiles of both directions staged by TMA (double-buffered), two
// columns per step in packed f32x2 arithmetic.
// ---------------------------------------------------------------------------
typedef unsigned long long f2x;
__device__ __forceinline__ f2x pk2(float a, float b)
{
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(f2x r, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); }
__device__ __forceinline__ f2x mul2(f2x a, f2x b)
{
    f2x d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x add2(f2x a, f2x b)
{
    f2x d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c)
{
    f2x d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__global__ void __launch_bounds__(CV_T) cv_loo_fast_kernel(const float2 *__restrict__ sc, int64_t N, int NT,
                                                           const uint2 *__restrict__ tile_u,
                                                           const uint32_t *__restrict__ perm, const int *argmin,
                                                           CvCands cc, double xs, float *loo, unsigned int *status,
                                                           unsigned wait_polls)
{
    __shared__ __align__(128) float2 buf[2][CV_T];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_stop;
    const int tid = threadIdx.x;
    const int a = blockIdx.x;
    const int best = *argmin;
    int cs = 0;
    for (int c = 0; c < cc.n; ++c)
        if (cc.orig[c] == best) cs = c;
    const float kc = cc.k[cs];
    const float kk = (float)(-2.0 * KDE_LOG2E) * kc;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_barrier_init();
    }
    __syncthreads();
    const int64_t i = (int64_t)a * CV_T + tid;
    const bool rvalid = i < N;
    const float2 me = sc[i];
    const uint2 ta = tile_u[a];
    const f2x mx = pk2(me.x, me.x), my = pk2(-me.y, -me.y), k2 = pk2(kk, kk);
    double sum = 0.0;
    Walk w{0, 0, 0};
    int b_cur = 0, d_cur = 0;
    bool have = walk_next(w, a, NT, tile_u, ta, kc, b_cur, d_cur);
    unsigned phase[2] = {0u, 0u};
    int cur = 0;
    if (have && tid == 0) tma_load_1d(buf[cur], sc + (size_t)b_cur * CV_T, CV_T * sizeof(float2), &bar[cur]);
    bool failed = false;
    while (have) {
        int b_nxt = 0, d_nxt = 0;
        const bool next = walk_next(w, a, NT, tile_u, ta, kc, b_nxt, d_nxt);
        if (next && tid == 0)
            tma_load_1d(buf[cur ^ 1], sc + (size_t)b_nxt * CV_T, CV_T * sizeof(float2), &bar[cur ^ 1]);
        if (!tile_wait(bar, phase, cur, next, wait_polls, &s_stop, status)) {
            failed = true;
            break;
        }
        const int64_t col0 = (int64_t)b_cur * CV_T;
        const int ncol = (int)(N - col0 < CV_T ? N - col0 : CV_T);
        const float2 *t = buf[cur];
        float tile_sum;
        if (d_cur == 0 || ncol < CV_T) {
            float acc = 0.f;
            for (int q = 0; q < ncol; ++q) {
                if (d_cur == 0 && q == tid) continue;
                const float2 o = t[q];
                const float s = me.x * o.y - me.y * o.x;
                acc += kde_ex2(s * s * kk);
            }
            tile_sum = acc;
        } else {
            const float4 *t4 = (const float4 *)t;
            f2x acc = pk2(0.f, 0.f);
#pragma unroll 4
            for (int q = 0; q < CV_T / 2; ++q) {
                const float4 o = t4[q];  // columns 2q and 2q+1: (sin, cos, sin, cos)
                const f2x sv = fma2(mx, pk2(o.y, o.w), mul2(my, pk2(o.x, o.z)));
                const f2x x = mul2(mul2(sv, sv), k2);
                float x0, x1;
                upk2(x, x0, x1);
                acc = add2(acc, pk2(kde_ex2(x0), kde_ex2(x1)));
            }
            float a0, a1;
            upk2(acc, a0, a1);
            tile_sum = a0 + a1;
        }
        sum += (double)tile_sum;
        __syncthreads();
        cur ^= 1;
        b_cur = b_nxt;
        d_cur = d_nxt;
        have = next;
    }
    if (failed) {
        if (tid == 0) kde_flag(status, KDE_DEV_WAIT_TIMEOUT, (unsigned)blockIdx.x);
        return;
    }
    if (!rvalid) return;
    const double v = xs * kde_norm((double)kc) * sum / (double)(N - 1);
    loo[perm ? perm[i] : i] = (float)v;
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
kde_status kde_cv_device(kde_ctx *ctx, const uint32_t *u, const float *kappa_rel, int64_t N, double L,
                         const double *cand_host, int n_cand, bool scale_mode, double *cv_dev, int *argmin_dev,
                         float *loo, double *kstar_dev)
{
    KdeRange r_cv("kdepic CV (pair sums, integral term, leave-one-out)");
    // candidates: internal ascending order
    CandList cl{};
    CvCands cc{};
    cl.n = cc.n = n_cand;
    cl.scale_mode = cc.scale_mode = scale_mode ? 1 : 0;
    std::vector<int> idx(n_cand);
    for (int c = 0; c < n_cand; ++c) idx[c] = c;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return cand_host[x] < cand_host[y]; });
    for (int c = 0; c < n_cand; ++c) {
        cl.k[c] = cand_host[idx[c]];
        cc.k[c] = (float)cand_host[idx[c]];
        cc.orig[c] = idx[c];
    }
    // bin sort (4096 bins at most; about 16 particles per bin)
    int nbins = 64;
    while (nbins < 4096 && (int64_t)nbins * 16 < N) nbins <<= 1;
    const int NT = (int)((N + CV_T - 1) / CV_T);
    const int64_t Np = (int64_t)NT * CV_T;
    uint32_t *us = (uint32_t *)kde_ws(ctx, WS_SORT_U, (size_t)Np * 4);
    uint32_t *perm = (uint32_t *)kde_ws(ctx, WS_SORT_PERM, (size_t)Np * 4);
    float *krs = scale_mode ? (float *)kde_ws(ctx, WS_SORT_P0, (size_t)Np * 4) : nullptr;
    float2 *sc = (float2 *)kde_ws(ctx, WS_CV_SC, (size_t)Np * sizeof(float2));
    uint2 *tile_u = (uint2 *)kde_ws(ctx, WS_CV_TILE, (size_t)NT * sizeof(uint2) + (size_t)NT * 4 + 64);
    float *tile_kmin = scale_mode ? (float *)(tile_u + NT) : nullptr;
    float *k2rel = scale_mode ? (float *)kde_ws(ctx, WS_CV_KR, (size_t)Np * 4) : nullptr;
    float *lnorm = scale_mode ? (float *)kde_ws(ctx, WS_CV_LNORM, (size_t)n_cand * N * 4) : nullptr;
    unsigned int *krmax = (unsigned int *)kde_ws(ctx, WS_WMAX, 64);  // [0] max, [1] min width bits
    double *f2 = (double *)kde_ws(ctx, WS_CV_F2, (size_t)n_cand * 8);
    double *tot = (double *)kde_ws(ctx, WS_CV_TOT, (size_t)n_cand * 8);
    if (!us || !perm || !sc || !tile_u || !krmax || !f2 || !tot || (scale_mode && (!krs || !k2rel || !lnorm)))
        return KDE_ENOMEM;
    SortPayload pl[1];
    int npl = 0;
    if (scale_mode) pl[npl++] = SortPayload{kappa_rel, krs, 4};
    KDE_TRY(kde_sort_by_bin(ctx, u, N, nbins, us, pl, npl, perm));
    KDE_CUDA(ctx, cudaMemsetAsync(krmax, 0, 4, ctx->stream), "kappa max memset");
    KDE_CUDA(ctx, cudaMemsetAsync(krmax + 1, 0x7f, 4, ctx->stream), "kappa min memset");
    int bin_shift = 32;
    for (int nb = nbins; nb > 1; nb >>= 1) --bin_shift;
    cv_prep_kernel<<<NT, CV_T, 0, ctx->stream>>>(us, krs, N, bin_shift, sc, tile_u, tile_kmin, k2rel, krmax, cl,
                                                  lnorm, ctx->d_status, ctx->norm_tab);
    KDE_LAUNCHED(ctx, "cv_prep_kernel");

    // pair totals
    int splits = 1;
    while ((int64_t)NT * splits < 2LL * ctx->sm_count && splits < NT) ++splits;
    const int nblocks = NT * splits;
    double *part = (double *)kde_ws(ctx, WS_CV_PART, (size_t)nblocks * n_cand * 8);
    if (!part) return KDE_ENOMEM;
    CvPairArgs A{};
    A.sc = sc;
    A.N = N;
    A.NT = NT;
    A.splits = splits;
    A.tile_u = tile_u;
    A.tile_kmin = tile_kmin;
    A.k2rel = k2rel;
    A.lnorm = lnorm;
    A.part = part;
    A.status = ctx->d_status;
    A.wait_polls = ctx->wait_polls;
    int nparts = nblocks;
    if (!scale_mode && n_cand <= CVF_MAXC) {
        // persistent fast path: enough work items for an even finish
        CvFast cf{};
        cf.n = n_cand;
        int ctas = 2 * ctx->sm_count;
        cf.splits = 1;
        while ((int64_t)NT * cf.splits < 8LL * ctas && cf.splits < NT) ++cf.splits;
        cf.nitems = NT * cf.splits;
        for (int c = 0; c < n_cand; ++c) {
            cf.k[c] = cc.k[c];
            cf.kk[c] = (float)(-2.0 * KDE_LOG2E) * cc.k[c];
        }
        for (int p = 0; p < CVF_MAXC / 2; ++p) {
            uint32_t lo, hi;
            memcpy(&lo, &cf.kk[2 * p], 4);
            memcpy(&hi, &cf.kk[2 * p + 1], 4);
            cf.kk2[p] = (kde_f2)lo | ((kde_f2)hi << 32);
        }
        part = (double *)kde_ws(ctx, WS_CV_PART, (size_t)cf.nitems * n_cand * 8 + 64);
        if (!part) return KDE_ENOMEM;
        int *counter = (int *)(part + (size_t)cf.nitems * n_cand);
        KDE_CUDA(ctx, cudaMemsetAsync(counter, 0, sizeof(int), ctx->stream), "cv counter memset");
        {
            KdeProfScope _ps(ctx, PROF_CV_PAIRS);
            cv_pairs_fast_kernel<<<ctas, CV_T, 0, ctx->stream>>>(sc, N, NT, tile_u, counter, part, ctx->d_status,
                                                                 ctx->wait_polls, cf);
        }
        KDE_LAUNCHED(ctx, "cv_pairs_fast_kernel");
        nparts = cf.nitems;
    } else {
        {
            KdeProfScope _ps(ctx, PROF_CV_PAIRS);
            if (scale_mode) cv_pairs_kernel<true><<<nblocks, CV_T, 0, ctx->stream>>>(A, cc);
            else cv_pairs_kernel<false><<<nblocks, CV_T, 0, ctx->stream>>>(A, cc);
        }
        KDE_LAUNCHED(ctx, "cv_pairs_kernel");
    }
    cv_reduce_kernel<<<n_cand, 256, 0, ctx->stream>>>(part, nparts, n_cand, tot);
    KDE_LAUNCHED(ctx, "cv_reduce_kernel");

    // integral term on fine grids
    {
        KdeRange r_("kdepic CV integral term");
        KDE_TRY(kde_cv_integral_term(ctx, us, N, krs, lnorm, krmax, cl, f2));
    }

    cv_combine_kernel<<<1, 32, 0, ctx->stream>>>(f2, tot, cc, cl, N, L, cv_dev, argmin_dev, kstar_dev);
    KDE_LAUNCHED(ctx, "cv_combine_kernel");

    // Leave-one-out densities at kappa* (uniform widths): the pair sums cost about
    // N^2 frac(kappa*) exponentials (frac = share of the circle inside the truncation
    // radius), the exact Fourier form about 4 N M(kappa*) exponential-equivalents.
    // The choice is made for the widest candidate and the narrowest: where the Fourier
    // form is cheaper at the largest candidate it is cheaper at every candidate.
    if (loo && !scale_mode) {
        const double kmx = cl.k[n_cand - 1];
        const double s2 = KDE_XCUT * KDE_LN2 / (2.0 * kmx);
        const double frac = s2 >= 1.0 ? 1.0 : 2.0 * asin(sqrt(s2)) / KDE_PI;
        if (4.0 * kde_spec_modes(kmx) < (double)N * frac) {
            KDE_TRY(kde_loo_spectral_device(ctx, u, N, L, cand_host, n_cand, argmin_dev, loo));
            return KDE_OK;
        }
    }
    if (loo) {
        CvLooArgs B{};
        B.sc = sc;
        B.N = N;
        B.NT = NT;
        B.tile_u = tile_u;
        B.tile_kmin = tile_kmin;
        B.k2rel = k2rel;
        B.lnorm = lnorm;
        B.perm = perm;
        B.argmin = argmin_dev;
        B.kr_bits = krmax;
        B.cc = cc;
        B.xs = KDE_TWO_PI / L;
        B.loo = loo;
        {
            KdeProfScope _ps(ctx, PROF_CV_LOO);
            if (scale_mode) cv_loo_kernel<true><<<NT, CV_T, 0, ctx->stream>>>(B);
            else
                cv_loo_fast_kernel<<<NT, CV_T, 0, ctx->stream>>>(sc, N, NT, tile_u, perm, argmin_dev, cc,
                                                                 KDE_TWO_PI / L, loo, ctx->d_status, ctx->wait_polls);
        }
        KDE_LAUNCHED(ctx, "cv_loo_kernel");
    }
    return KDE_OK;
}

// cost rule between the two exact forms of a uniform-width CV curve: pair sums
// cost about N^2 frac(kappa_c) / 2 exponentials per candidate (frac = share of
// the circle inside the truncation radius), the Fourier form about 4 N M(kappa_max)
// exponential-equivalents for the structure factor shared by all candidates
bool kde_cv_prefer_spectral(int64_t N, const double *cand, int n_cand)
{
    double kmax = 0.0, sfrac = 0.0;
    for (int c = 0; c < n_cand; ++c) {
        kmax = cand[c] > kmax ? cand[c] : kmax;
        const double s2 = KDE_XCUT * KDE_LN2 / (2.0 * cand[c]);
        sfrac += s2 >= 1.0 ? 1.0 : 2.0 * asin(sqrt(s2)) / KDE_PI;
    }
    return 8.0 * (double)kde_spec_modes(kmax) < (double)N * sfrac;
}

extern "C" kde_status kde_cv(kde_ctx *ctx, const uint32_t *u, const float *kappa_rel, int64_t N, double L,
                             const double *cand, int32_t n_cand, double *cv_out, int32_t *argmin_out, float *loo_out,
                             uint32_t flags)
{
    if (!ctx) return KDE_EINVAL;
    const bool scale = (flags & KDE_CV_SCALE) != 0;
    bool spectral = (flags & KDE_CV_SPECTRAL) != 0;
    const bool pairs = (flags & KDE_CV_PAIRS) != 0;
    if (flags & ~(KDE_CV_SCALE | KDE_CV_SPECTRAL | KDE_CV_PAIRS))
        return kde_fail(ctx, KDE_ENOTSUP, "kde_cv: unsupported flags 0x%x", flags);
    if (scale && spectral)
        return kde_fail(ctx, KDE_ENOTSUP, "kde_cv: the spectral form is for uniform candidate widths");
    if (spectral && pairs)
        return kde_fail(ctx, KDE_EINVAL, "kde_cv: KDE_CV_SPECTRAL and KDE_CV_PAIRS exclude each other");
    if (N < 2 || N > 0xFFFFFFFFll || !(L > 0) || !u || !cand || !cv_out || n_cand < 1 || n_cand > CV_MAXC)
        return kde_fail(ctx, KDE_EINVAL, "kde_cv: need 2 <= N < 2^32, L > 0, 1 <= n_cand <= %d, non-null arrays",
                        CV_MAXC);
    if (scale && !kappa_rel) return kde_fail(ctx, KDE_EINVAL, "kde_cv: KDE_CV_SCALE needs kappa_rel");
    for (int c = 0; c < n_cand; ++c)
        if (!(cand[c] > 0 && cand[c] <= KDE_KAPPA_MAX))
            return kde_fail(ctx, KDE_EINVAL, "kde_cv: candidate %d = %g outside (0, 1e6]", c, cand[c]);
    if (!scale && !pairs && !spectral) spectral = kde_cv_prefer_spectral(N, cand, n_cand);
    cudaSetDevice(ctx->device);
    double *cvd = (double *)kde_ws(ctx, WS_CV_OUT, (size_t)n_cand * 8 + 64);
    if (!cvd) return KDE_ENOMEM;
    int *amin = (int *)(cvd + n_cand);
    if (spectral) KDE_TRY(kde_cv_spectral_device(ctx, u, N, L, cand, n_cand, cvd, amin, loo_out, nullptr));
    else
        KDE_TRY(kde_cv_device(ctx, u, scale ? kappa_rel : nullptr, N, L, cand, n_cand, scale, cvd, amin, loo_out,
                              nullptr));
    KDE_CUDA(ctx, cudaMemcpyAsync(cv_out, cvd, (size_t)n_cand * 8, cudaMemcpyDeviceToHost, ctx->stream), "cv copy");
    int am = 0;
    KDE_CUDA(ctx, cudaMemcpyAsync(&am, amin, 4, cudaMemcpyDeviceToHost, ctx->stream), "argmin copy");
    KDE_TRY(kde_sync(ctx));
    if (argmin_out) *argmin_out = am;
    return KDE_OK;
}

// ---------------------------------------------------------------------------
// Silverman particle-wise widths (Sec. II.C)
// ---------------------------------------------------------------------------
#define AD_BLOCKS 256
// scalars of the Silverman step: K0 = (2 pi / L) norm(kappa*) (the kernel's value at its
// own particle), kappa*, the log-mean of the pilot, and the FP32 forms of the pilot's
// coefficients f = a loo + b, a = (n - 1) / n, b = K0 / n.  Worked out once by one
// thread (the FP64 Bessel series is slow on this part), read by every thread after.
struct AdaptPar {
    double K0, ks, logg;
    float a, b, ks_f, logg_f;
};

__global__ void adapt_par_kernel(int64_t N, double xs, const double *kstar_dev, double kstar_h, AdaptPar *P)
{
    const double ks = kstar_dev ? *kstar_dev : kstar_h, n = (double)N;
    const double K0 = xs * kde_norm(ks);
    P->K0 = K0;
    P->ks = ks;
    P->a = (float)((n - 1.0) / n);
    P->b = (float)(K0 / n);
    P->ks_f = (float)ks;
}

// log-mean of the pilot: after the block partials of adapt_logsum_dev_kernel, one block
// adds them by a fixed tree
__global__ void __launch_bounds__(256) adapt_mean_kernel(const double *part, int64_t N, AdaptPar *P)
{
    __shared__ double red[AD_BLOCKS];
    red[threadIdx.x] = part[threadIdx.x];
    __syncthreads();
    for (int o = AD_BLOCKS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        P->logg = red[0] / (double)N;
        P->logg_f = (float)P->logg;
    }
}

template <typename T>
__global__ void adapt_apply_kernel(const float *loo, int64_t N, const AdaptPar *__restrict__ P, double alpha,
                                   double kmin, double kmax, T *kappa_out, T *norm_out, const float2 *ntab)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    // lambda = (f/g)^-alpha, kappa = kappa* / lambda^2; FP32 widths in FP32 with base-2
    // logarithms (the log-mean of adapt_logsum_dev_kernel<true> is in the same base), FP64
    // widths in FP64 with natural ones
    T k;
    if constexpr (sizeof(T) == 4) {
        const float f = fmaf(P->a, loo[i], P->b);
        float kf = P->ks_f * exp2f((float)(2.0 * alpha) * (log2f(f) - P->logg_f));
        kf = kf < (float)kmin ? (float)kmin : (kf > (float)kmax ? (float)kmax : kf);
        k = kf;
    } else {
        const double n = (double)N;
        const double f = ((n - 1.0) * (double)loo[i] + P->K0) / n;
        double kd = P->ks * exp(2.0 * alpha * (log(f) - P->logg));
        kd = kd < kmin ? kmin : (kd > kmax ? kmax : kd);
        k = kd;
    }
    kappa_out[i] = k;
    if (norm_out) {
        // FP32 widths take the tabulated norm, FP64 widths the FP64 Bessel series
        if constexpr (sizeof(T) == 4) norm_out[i] = (T)kde_norm_tab(ntab, (float)k);
        else norm_out[i] = (T)kde_norm((double)k);
    }
}

// block partials of the pilot's log-sum.  F32: base-2 logarithms of the FP32 pilot,
// added in FP32 in runs of 16 and the runs in FP64, for FP32 widths; otherwise natural
// FP64 logarithms of the FP64 pilot
template <bool F32>
__global__ void adapt_logsum_dev_kernel(const float *loo, int64_t N, const AdaptPar *__restrict__ P, double *part)
{
    __shared__ double red[256];
    const double n = (double)N;
    double s = 0.0;
    float fs = 0.f;
    int run = 0;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)AD_BLOCKS * 256) {
        if (F32) {
            fs += log2f(fmaf(P->a, loo[i], P->b));
            if (++run == 16) {
                s += (double)fs;
                fs = 0.f;
                run = 0;
            }
        } else {
            s += log(((n - 1.0) * (double)loo[i] + P->K0) / n);
        }
    }
    s += (double)fs;
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

kde_status kde_adapt_device(kde_ctx *ctx, const float *loo, int64_t N, double L, const double *kstar_dev,
                            double kstar_host, double alpha, double kmin, double kmax, void *kappa_out,
                            void *norm_out, bool f64)
{
    double *part = (double *)kde_ws(ctx, WS_CV_RED, AD_BLOCKS * 8 + sizeof(AdaptPar) + 64);
    if (!part) return KDE_ENOMEM;
    AdaptPar *P = (AdaptPar *)(part + AD_BLOCKS);
    const double xs = KDE_TWO_PI / L;
    adapt_par_kernel<<<1, 1, 0, ctx->stream>>>(N, xs, kstar_dev, kstar_host, P);
    KDE_LAUNCHED(ctx, "adapt_par_kernel");
    if (f64) adapt_logsum_dev_kernel<false><<<AD_BLOCKS, 256, 0, ctx->stream>>>(loo, N, P, part);
    else adapt_logsum_dev_kernel<true><<<AD_BLOCKS, 256, 0, ctx->stream>>>(loo, N, P, part);
    KDE_LAUNCHED(ctx, "adapt_logsum_dev_kernel");
    adapt_mean_kernel<<<1, AD_BLOCKS, 0, ctx->stream>>>(part, N, P);
    KDE_LAUNCHED(ctx, "adapt_mean_kernel");
    unsigned grid = (unsigned)((N + 255) / 256);
    if (f64)
        adapt_apply_kernel<double><<<grid, 256, 0, ctx->stream>>>(loo, N, P, alpha, kmin, kmax, (double *)kappa_out,
                                                                   (double *)norm_out, ctx->norm_tab);
    else
        adapt_apply_kernel<float><<<grid, 256, 0, ctx->stream>>>(loo, N, P, alpha, kmin, kmax, (float *)kappa_out,
                                                                  (float *)norm_out, ctx->norm_tab);
    KDE_LAUNCHED(ctx, "adapt_apply_kernel");
    return KDE_OK;
}

extern "C" kde_status kde_adapt_widths(kde_ctx *ctx, const float *loo, int64_t N, double L, double kappa_star,
                                       double alpha, double kappa_min, double kappa_max, float *kappa_out)
{
    if (!ctx) return KDE_EINVAL;
    if (N < 2 || !loo || !kappa_out || !(L > 0) || !(kappa_star > 0 && kappa_star <= KDE_KAPPA_MAX) ||
        !(alpha >= 0) || !(kappa_min <= kappa_max))
        return kde_fail(ctx, KDE_EINVAL, "kde_adapt_widths: bad arguments");
    cudaSetDevice(ctx->device);
    return kde_adapt_device(ctx, loo, N, L, nullptr, kappa_star, alpha, kappa_min, kappa_max, kappa_out, nullptr,
                            false);
}

// ---------------------------------------------------------------------------
// CV of the first-order (CIC) shape's width (Sec. IV, Fig. compare_high_order f):
// S_h(x) = (1/h) B_1(x/h), and int fhat^2 = (1/n^2) sum_{i,j} (1/h) B_3((x_i - x_j)/h)
// since B_1 * B_1 = B_3.  Both sums have compact support (|d| < h and < 2h), so
// the bin-sorted tiles are walked only while their gap is below 2 h_max; pair
// distances come from exact integer code differences.  Unordered tile pairs,
// FP32 sums per tile, FP64 per CTA, a fixed reduction order.
// ---------------------------------------------------------------------------
#define CIC_MAXC 64
#define CIC_G 8

struct CicCands {
    int n;
    float inv_h[CIC_MAXC];  // 1 / h_c in position-code units
};

// the tile walk of walk_next with an integer gap threshold (codes)
__device__ __forceinline__ bool walk_next_gap(Walk &w, int a, int NT, const uint2 *tile_u, uint2 ta, uint32_t reach,
                                              int &b, int &d)
{
    for (;;) {
        if (w.phase == 0) {
            if (w.k >= NT) {
                w.phase = 2;
                return false;
            }
            const int bb = (a + w.k) % NT;
            if (w.k == 0 || tile_gap(ta, tile_u[bb]) <= reach) {
                b = bb;
                d = w.k;
                w.F = w.k;
                ++w.k;
                return true;
            }
            w.phase = 1;
            w.k = 1;
        } else if (w.phase == 1) {
            if (w.k >= NT - w.F) {
                w.phase = 2;
                return false;
            }
            const int bb = ((a - w.k) % NT + NT) % NT;
            if (tile_gap(ta, tile_u[bb]) <= reach) {
                b = bb;
                d = -w.k;
                ++w.k;
                return true;
            }
            w.phase = 2;
            return false;
        } else {
            return false;
        }
    }
}

// per row tile: sums over ordered pairs i != j of B_1(d / h_c) and B_3(d / h_c)
// (part[a][c] and part[a][n + c])
__global__ void __launch_bounds__(CV_T)
    cv_cic_kernel(const uint32_t *__restrict__ us, int64_t N, int NT, const uint2 *__restrict__ tile_u, uint32_t reach,
                  CicCands cc, double *part)
{
    __shared__ uint32_t cu[CV_T];
    __shared__ double wacc[CV_WARPS][2 * CIC_MAXC];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int a = blockIdx.x;
    const int64_t i = (int64_t)a * CV_T + tid;
    const bool rvalid = i < N;
    const uint32_t ui = rvalid ? us[i] : 0u;
    for (int c = tid; c < CV_WARPS * 2 * CIC_MAXC; c += CV_T) (&wacc[0][0])[c] = 0.0;
    const uint2 ta = tile_u[a];
    Walk w{0, 0, 0};
    int b = 0, d = 0;
    while (walk_next_gap(w, a, NT, tile_u, ta, reach, b, d)) {
        if (!canonical_pair(a, b, NT)) continue;
        const int64_t col0 = (int64_t)b * CV_T;
        const int ncol = (int)(N - col0 < CV_T ? N - col0 : CV_T);
        __syncthreads();  // the previous tile's readers are done
        if (tid < ncol) cu[tid] = us[col0 + tid];
        __syncthreads();
        const bool diag = d == 0;
        const float wgt = diag ? 1.0f : 2.0f;
        for (int cg = 0; cg < cc.n; cg += CIC_G) {
            float s1[CIC_G], s3[CIC_G];
#pragma unroll
            for (int k = 0; k < CIC_G; ++k) s1[k] = s3[k] = 0.f;
            for (int q = 0; q < ncol; ++q) {
                if (diag && q == tid) continue;
                const uint32_t dd = cu[q] - ui;
                const float dist = (float)(dd < 0x80000000u ? dd : 0u - dd);
#pragma unroll
                for (int k = 0; k < CIC_G; ++k) {
                    const float t = dist * cc.inv_h[cg + k < cc.n ? cg + k : cc.n - 1];
                    const float b1 = fmaxf(0.f, 1.f - t), b2 = fmaxf(0.f, 2.f - t);
                    s1[k] += b1;
                    s3[k] += (b2 * b2 * b2 - 4.f * b1 * b1 * b1) * (1.f / 6.f);
                }
            }
#pragma unroll
            for (int k = 0; k < CIC_G; ++k) {
                float v1 = rvalid ? s1[k] : 0.f, v3 = rvalid ? s3[k] : 0.f;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    v1 += __shfl_xor_sync(0xffffffffu, v1, o);
                    v3 += __shfl_xor_sync(0xffffffffu, v3, o);
                }
                if (lane == 0 && cg + k < cc.n) {
                    wacc[warp][cg + k] += (double)wgt * (double)v1;
                    wacc[warp][cc.n + cg + k] += (double)wgt * (double)v3;
                }
            }
        }
    }
    __syncthreads();
    for (int c = tid; c < 2 * cc.n; c += CV_T) {
        double s = 0.0;
        for (int ww = 0; ww < CV_WARPS; ++ww) s += wacc[ww][c];
        part[(size_t)a * 2 * cc.n + c] = s;
    }
}

// CV_c = (n B_3(0) + S3_c) / (n^2 h_c) - 2 S1_c / (n (n - 1) h_c), x units; argmin
// (smallest index on ties)
__global__ void cic_combine_kernel(const double *tot, int n_cand, int64_t N, CandList hl, double *cv, int *argmin)
{
    if (threadIdx.x != 0) return;
    const double n = (double)N;
    for (int c = 0; c < n_cand; ++c) {
        const double h = hl.k[c];
        cv[c] = (n * (2.0 / 3.0) + tot[n_cand + c]) / (n * n * h) - 2.0 * tot[c] / (n * (n - 1.0) * h);
    }
    int best = 0;
    for (int c = 1; c < n_cand; ++c)
        if (cv[c] < cv[best]) best = c;
    *argmin = best;
}

extern "C" kde_status kde_cv_cic(kde_ctx *ctx, const uint32_t *u, int64_t N, double L, const double *h_cand,
                                 int32_t n_cand, double *cv_out, int32_t *argmin_out)
{
    if (!ctx) return KDE_EINVAL;
    if (N < 2 || N > 0xFFFFFFFFll || !u || !(L > 0) || !h_cand || n_cand < 1 || n_cand > CIC_MAXC || !cv_out)
        return kde_fail(ctx, KDE_EINVAL, "kde_cv_cic: need 2 <= N < 2^32, L > 0, 1 <= n_cand <= %d, non-null arrays",
                        CIC_MAXC);
    double hmax = 0.0;
    CicCands cc{};
    CandList hl{};
    cc.n = hl.n = n_cand;
    for (int c = 0; c < n_cand; ++c) {
        if (!(h_cand[c] > 0 && 4.0 * h_cand[c] < L))
            return kde_fail(ctx, KDE_EINVAL, "kde_cv_cic: candidate %d needs 0 < h < L/4", c);
        hmax = h_cand[c] > hmax ? h_cand[c] : hmax;
        cc.inv_h[c] = (float)(L / 4294967296.0 / h_cand[c]);
        hl.k[c] = h_cand[c];
    }
    cudaSetDevice(ctx->device);
    int nbins = 64;
    while (nbins < 4096 && (int64_t)nbins * 16 < N) nbins <<= 1;
    const int NT = (int)((N + CV_T - 1) / CV_T);
    const int64_t Np = (int64_t)NT * CV_T;
    uint32_t *us = (uint32_t *)kde_ws(ctx, WS_SORT_U, (size_t)Np * 4);
    float2 *sc = (float2 *)kde_ws(ctx, WS_CV_SC, (size_t)Np * sizeof(float2));
    uint2 *tile_u = (uint2 *)kde_ws(ctx, WS_CV_TILE, (size_t)NT * sizeof(uint2) + (size_t)NT * 4 + 64);
    double *part = (double *)kde_ws(ctx, WS_CV_PART, (size_t)NT * 2 * n_cand * 8);
    double *tot = (double *)kde_ws(ctx, WS_CV_TOT, (size_t)2 * n_cand * 8);
    double *cvd = (double *)kde_ws(ctx, WS_CV_OUT, (size_t)n_cand * 8 + 64);
    if (!us || !sc || !tile_u || !part || !tot || !cvd) return KDE_ENOMEM;
    int *amin = (int *)(cvd + n_cand);
    KDE_TRY(kde_sort_by_bin(ctx, u, N, nbins, us, nullptr, 0, nullptr));
    int bin_shift = 32;
    for (int nb = nbins; nb > 1; nb >>= 1) --bin_shift;
    cv_prep_kernel<<<NT, CV_T, 0, ctx->stream>>>(us, nullptr, N, bin_shift, sc, tile_u, nullptr, nullptr, nullptr,
                                                  CandList{}, nullptr, ctx->d_status, ctx->norm_tab);
    KDE_LAUNCHED(ctx, "cv_prep_kernel");
    const double reach_d = 2.0 * hmax / L * 4294967296.0;  // B_3 support in codes
    const uint32_t reach = reach_d >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)ceil(reach_d);
    {
        KdeProfScope _ps(ctx, PROF_CV_PAIRS);
        cv_cic_kernel<<<NT, CV_T, 0, ctx->stream>>>(us, N, NT, tile_u, reach, cc, part);
    }
    KDE_LAUNCHED(ctx, "cv_cic_kernel");
    cv_reduce_kernel<<<2 * n_cand, 256, 0, ctx->stream>>>(part, NT, 2 * n_cand, tot);
    KDE_LAUNCHED(ctx, "cv_reduce_kernel");
    cic_combine_kernel<<<1, 32, 0, ctx->stream>>>(tot, n_cand, N, hl, cvd, amin);
    KDE_LAUNCHED(ctx, "cic_combine_kernel");
    KDE_CUDA(ctx, cudaMemcpyAsync(cv_out, cvd, (size_t)n_cand * 8, cudaMemcpyDeviceToHost, ctx->stream), "cv copy");
    int am = 0;
    KDE_CUDA(ctx, cudaMemcpyAsync(&am, amin, 4, cudaMemcpyDeviceToHost, ctx->stream), "argmin copy");
    KDE_TRY(kde_sync(ctx));
    if (argmin_out) *argmin_out = am;
    return KDE_OK;
}
