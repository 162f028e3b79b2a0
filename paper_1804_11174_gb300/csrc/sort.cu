// sort.cu -- stable counting sort of particles by bin (cell) index.
//
// A block of wpb warps owns a tile of wpb * unit particles; warp w of the block
// owns the w-th contiguous unit of the tile (unit a multiple of 32).
//   count   : the block's histogram of its tile (keys shared by several lanes of a
//             warp are added once, by their leader) -> counts[bin][block]
//             (bin-major, so that the destination order of the tiles' segments is
//             the flat index bin * nblocks + block)
//   scan    : exclusive scan of each 2048-entry tile of the flat counts array in place,
//             plus the tile totals, and zeroing of the second count table; every
//             scatter block scans the (few) tile totals itself, so no block waits for
//             another.
//   scatter : each warp histograms its unit in shared memory, the block turns the
//             warps' histograms into destination starts (its segment start plus the
//             counts of the earlier warps), then every warp ranks equal keys in each
//             32-particle step with __match_any_sync and writes every particle
//             (position and payloads) to its start + rank.
// In the PIC step the count pass is skipped when the previous step's gather + push
// kernel has already added the new positions' counts into the table the previous
// scan zeroed (two tables, used in turn).  The scan and the scatter are launched as
// programmatic dependents: the scatter's key loads and histograms overlap the scan.
// The order inside a bin is the input order (stable), so results are
// deterministic.  The count table has one entry per (bin, block) rather than per
// (bin, warp), so it stays small next to the particle data.
//
// The same kernels in digit mode (key = a bit field of the code) give an LSD
// radix sort of the full 32-bit codes: four stable passes of 8-bit digits.
#include "common.cuh"

#define SORT_MAX_COUNTS (1 << 22)
#define SCAN_TILE 2048
#define SCAN_THREADS 256

__device__ __forceinline__ int bin_of(uint32_t u, int nbins) { return (int)(((uint64_t)u * (uint64_t)nbins) >> 32); }

// sort key: the bin floor(u nbins / 2^32), or in digit mode the bit field
// (u >> shift) mod nbins (nbins a power of two)
template <bool DIGIT>
__device__ __forceinline__ int sort_key(uint32_t u, int nbins, int shift)
{
    if (DIGIT) return (int)((u >> shift) & (uint32_t)(nbins - 1));
    return bin_of(u, nbins);
}

#define SORT_MAXR 4  // 32-particle steps whose loads are issued together (8-byte payloads)
#define SORT_MAXR_N 8  // the same with 4-byte payloads only
#define COUNT_MAXR 8  // the same for the count kernel

// the block's histogram of its tile; each thread issues the loads of COUNT_MAXR
// steps before it uses any of them
template <bool DIGIT>
__global__ void sort_count_kernel(const uint32_t *__restrict__ u, int64_t N, int nbins, int shift, int unit,
                                  int nblk, unsigned int *counts)
{
    extern __shared__ unsigned int hist[];
    const int lane = threadIdx.x & 31;
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const int64_t tile = (int64_t)(blockDim.x >> 5) * unit;
    const int64_t t0 = (int64_t)blockIdx.x * tile, t1 = t0 + tile < N ? t0 + tile : N;
    for (int64_t c0 = t0 + (threadIdx.x & ~31); c0 < t1; c0 += (int64_t)blockDim.x * COUNT_MAXR) {
        uint32_t uu[COUNT_MAXR];
#pragma unroll
        for (int r = 0; r < COUNT_MAXR; ++r) {
            const int64_t i = c0 + (int64_t)r * blockDim.x + lane;
            uu[r] = i < t1 ? u[i] : 0u;
        }
#pragma unroll
        for (int r = 0; r < COUNT_MAXR; ++r) {
            const int64_t i = c0 + (int64_t)r * blockDim.x + lane;
            const int key = i < t1 ? sort_key<DIGIT>(uu[r], nbins, shift) : -1;
            const unsigned int peers = __match_any_sync(0xffffffffu, key);
            if (key >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[key], (unsigned int)__popc(peers));
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) counts[(size_t)b * nblk + blockIdx.x] = hist[b];
}

// exclusive scan of each SCAN_TILE-element tile in place: each thread scans a run of
// SCAN_TILE / SCAN_THREADS consecutive entries in registers (16-byte loads and stores
// where aligned), then one block scan of the run totals; the tile totals go to tot.  The
// scatter scans the (few) tile totals itself, so no block waits for another.
__global__ void __launch_bounds__(SCAN_THREADS) sort_scan_kernel(unsigned int *a, int64_t n, unsigned int *tot,
                                                                 unsigned int *zero_out)
{
    constexpr int R = SCAN_TILE / SCAN_THREADS;  // consecutive entries a thread
    __shared__ unsigned int wsum[SCAN_THREADS / 32];
    kde_pdl_wait();  // the counts come from the kernel before
    kde_pdl_trigger();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i0 = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)tid * R;
    // vector loads and stores where the run is whole and 16-byte aligned
    const bool vec = i0 + R <= n && ((uintptr_t)(a + i0) & 15u) == 0;
    unsigned int v[R];
    if (vec) {
#pragma unroll
        for (int q = 0; q < R / 4; ++q) {
            const uint4 w = reinterpret_cast<const uint4 *>(a + i0)[q];
            v[4 * q] = w.x;
            v[4 * q + 1] = w.y;
            v[4 * q + 2] = w.z;
            v[4 * q + 3] = w.w;
        }
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = i0 + r < n ? a[i0 + r] : 0u;
    }
    // the thread's run scanned in registers, then one block scan of the run totals
    unsigned int run = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const unsigned int x = v[r];
        v[r] = run;
        run += x;
    }
    unsigned int inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    unsigned int woff = 0, total = 0;
#pragma unroll
    for (int w = 0; w < SCAN_THREADS / 32; ++w) {
        woff += w < warp ? wsum[w] : 0u;
        total += wsum[w];
    }
    const unsigned int base = woff + inc - run;
    if (vec) {
#pragma unroll
        for (int q = 0; q < R / 4; ++q)
            reinterpret_cast<uint4 *>(a + i0)[q] =
                make_uint4(base + v[4 * q], base + v[4 * q + 1], base + v[4 * q + 2], base + v[4 * q + 3]);
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (i0 + r < n) a[i0 + r] = base + v[r];
    }
    if (tid == 0) tot[blockIdx.x] = total;
    // the next step's count table (added to by the PIC gather) starts from zero
    if (zero_out) {
        if (i0 + R <= n && ((uintptr_t)(zero_out + i0) & 15u) == 0) {
#pragma unroll
            for (int q = 0; q < R / 4; ++q) reinterpret_cast<uint4 *>(zero_out + i0)[q] = make_uint4(0u, 0u, 0u, 0u);
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (i0 + r < n) zero_out[i0 + r] = 0u;
        }
    }
}

struct ScatterPl {
    const void *src[4];
    void *dst[4];
    int elem[4];
    int n;
};

// NPL payload arrays (4- or 8-byte elements) move with the keys.  NARROW (every payload
// 4 bytes) takes SORT_MAXR_N steps of 32 particles a chunk, else SORT_MAXR.  A warp
// whose unit fits one chunk loads its keys and payloads once, at the start, and keeps
// them in registers through the ranking: every load of the kernel is then in flight
// before the first dependent step, and the whole pass is one round of loads, the
// block's offsets and one round of stores.  With a larger unit the payloads are
// loaded chunk by chunk in the write phase.  The keys are the sort's input, which
// the scan does not write, so they are read before kde_pdl_wait(); the scan's
// offsets and tile totals after it.
template <bool DIGIT, int NPL, bool NARROW>
__global__ void __launch_bounds__(256, NARROW ? 4 : 1) sort_scatter_kernel(const uint32_t *__restrict__ u, int64_t N, int nbins,
                                                           int shift, int unit, int nblk,
                                                           const unsigned int *__restrict__ seg,
                                                           const unsigned int *__restrict__ tot, int ntiles,
                                                           uint32_t *u_out, ScatterPl pl, uint32_t *perm_out)
{
    constexpr int SR = NARROW ? SORT_MAXR_N : SORT_MAXR;
    constexpr int NP1 = NPL > 0 ? NPL : 1;
    extern __shared__ unsigned int hist[];
    const int wpb = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned int *h = hist + (size_t)warp * nbins;
    unsigned int *tpre = hist + (size_t)wpb * nbins;  // exclusive prefix of the scan's tile totals
    for (int b = threadIdx.x; b < wpb * nbins; b += blockDim.x) hist[b] = 0;
    const int64_t i0 = ((int64_t)blockIdx.x * wpb + warp) * unit;
    const int64_t i1 = i0 + unit < N ? i0 + unit : N;  // empty when i0 >= N
    const bool one = i1 - i0 <= 32 * SR;               // the unit is a single chunk
    const unsigned int lt = (1u << lane) - 1u;
    uint32_t uu[SR];
    uint32_t lo[NP1][SR], hi[NARROW ? 1 : NP1][SR];
    auto load_payload = [&](int64_t c0) {
#pragma unroll
        for (int r = 0; r < SR; ++r) {
            const int64_t i = c0 + r * 32 + lane;
            const bool ok = i < i1;
#pragma unroll
            for (int k = 0; k < NPL; ++k) {
                if (!NARROW && pl.elem[k] == 8) {
                    const uint2 w = ok ? ((const uint2 *)pl.src[k])[i] : make_uint2(0u, 0u);
                    lo[k][r] = w.x;
                    hi[NARROW ? 0 : k][r] = w.y;
                } else {
                    lo[k][r] = ok ? ((const uint32_t *)pl.src[k])[i] : 0u;
                }
            }
        }
    };
    __syncthreads();
    // per-warp histograms of the keys
    for (int64_t c0 = i0; c0 < i1; c0 += 32 * SR) {
#pragma unroll
        for (int r = 0; r < SR; ++r) {
            const int64_t i = c0 + r * 32 + lane;
            uu[r] = i < i1 ? u[i] : 0u;
        }
        if (one) load_payload(c0);
#pragma unroll
        for (int r = 0; r < SR; ++r) {
            const int64_t i = c0 + r * 32 + lane;
            const int key = i < i1 ? sort_key<DIGIT>(uu[r], nbins, shift) : -1;
            const unsigned int peers = __match_any_sync(0xffffffffu, key);
            if (key >= 0 && lane == __ffs(peers) - 1) h[key] += __popc(peers);
            __syncwarp();
        }
    }
    kde_pdl_wait();  // the scan's results from here on
    kde_pdl_trigger();
    if (warp == 0) {
        unsigned int carry = 0;
        for (int t0 = 0; t0 < ntiles; t0 += 32) {
            const unsigned int x = t0 + lane < ntiles ? tot[t0 + lane] : 0u;
            unsigned int inc = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (t0 + lane < ntiles) tpre[t0 + lane] = carry + inc - x;
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
    }
    __syncthreads();
    // destination starts: the block's segment start of each bin plus the earlier warps'
    // counts
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        const size_t flat = (size_t)b * nblk + blockIdx.x;
        unsigned int run = seg[flat] + tpre[flat / SCAN_TILE];
        for (int w = 0; w < wpb; ++w) {
            const unsigned int t = hist[(size_t)w * nbins + b];
            hist[(size_t)w * nbins + b] = run;
            run += t;
        }
    }
    __syncthreads();
    for (int64_t c0 = i0; c0 < i1; c0 += 32 * SR) {
        if (!one) {
#pragma unroll
            for (int r = 0; r < SR; ++r) {
                const int64_t i = c0 + r * 32 + lane;
                uu[r] = i < i1 ? u[i] : 0u;
            }
            load_payload(c0);
        }
#pragma unroll
        for (int r = 0; r < SR; ++r) {
            const int64_t i = c0 + r * 32 + lane;
            if (c0 + r * 32 >= i1) break;
            const bool valid = i < i1;
            const int key = valid ? sort_key<DIGIT>(uu[r], nbins, shift) : -1;
            const unsigned int peers = __match_any_sync(0xffffffffu, key);
            const unsigned int rank = __popc(peers & lt);
            const unsigned int before = valid ? h[key] : 0u;
            __syncwarp();
            if (valid && rank == 0) h[key] = before + __popc(peers);
            __syncwarp();
            // a count table that disagreed with the keys could not send a write past the arrays
            const unsigned int dst = min(before + rank, (unsigned int)(N - 1));
            if (valid) {
                u_out[dst] = uu[r];
#pragma unroll
                for (int k = 0; k < NPL; ++k) {
                    if (!NARROW && pl.elem[k] == 8) ((uint2 *)pl.dst[k])[dst] = make_uint2(lo[k][r], hi[NARROW ? 0 : k][r]);
                    else ((uint32_t *)pl.dst[k])[dst] = lo[k][r];
                }
                if (perm_out) perm_out[dst] = (uint32_t)i;
            }
        }
    }
}

template <bool DIGIT, int NPL, bool NARROW>
static cudaError_t scatter_launch(kde_ctx *ctx, int nblk, int threads, size_t smem, const uint32_t *u, int64_t N,
                                  int nbins, int shift, int unit, const unsigned int *seg, const unsigned int *tot,
                                  int ntiles, uint32_t *u_out, const ScatterPl &sp, uint32_t *perm_out)
{
    auto kern = sort_scatter_kernel<DIGIT, NPL, NARROW>;
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    return kde_launch(ctx, true, kern, dim3(nblk), dim3(threads), smem, u, N, nbins, shift, unit, nblk, seg, tot,
                      ntiles, u_out, sp, perm_out);
}

// tile geometry of a sort of N keys into nbins bins: wpb warps of `unit` keys a block
static void sort_geometry(int64_t N, int nbins, int &wpb, int &unit, int &nblk)
{
    // the scatter keeps wpb warp-private histograms of nbins entries and the scan's tile
    // totals (one per SCAN_TILE count entries) in at most 100 KB of shared memory, and the
    // count table has at most SORT_MAX_COUNTS entries: fewer warps a block for many bins,
    // then longer units until both hold
    wpb = 8;
    while (wpb > 1 && (size_t)wpb * nbins * 4 > 96 * 1024) wpb >>= 1;
    unit = 256;
    for (;;) {
        const int64_t tile = (int64_t)wpb * unit;
        const int64_t nb = (N + tile - 1) / tile;
        const int64_t ncounts = (int64_t)nbins * nb;
        const int64_t ntiles = (ncounts + SCAN_TILE - 1) / SCAN_TILE;
        if (ncounts <= SORT_MAX_COUNTS && (int64_t)wpb * nbins * 4 + ntiles * 4 <= 100 * 1024) {
            nblk = (int)nb;
            return;
        }
        unit *= 2;
    }
}

// the two count tables of the PIC step (one consumed by this step's sort while the
// gather adds the next step's into the other), in one workspace slot
static unsigned int *count_tables(kde_ctx *ctx, int64_t ncounts)
{
    return (unsigned int *)kde_ws(ctx, WS_SORT_COUNTS, (size_t)ncounts * 8);
}

kde_status kde_sort_counts_table(kde_ctx *ctx, int64_t N, int nbins, SortCounts *out)
{
    int wpb, unit, nblk;
    sort_geometry(N, nbins, wpb, unit, nblk);
    int sh = 0;
    while ((1LL << sh) < (int64_t)wpb * unit) ++sh;
    const int64_t ncounts = (int64_t)nbins * nblk;
    unsigned int *counts = count_tables(ctx, ncounts);
    if (!counts) return KDE_ENOMEM;
    out->counts = counts + (ctx->count_flip ? ncounts : 0);  // the table the next sort reads
    out->nblk = nblk;
    out->tile_shift = sh;
    return KDE_OK;
}

template <bool DIGIT>
static kde_status sort_pass(kde_ctx *ctx, const uint32_t *u, int64_t N, int nbins, int shift, uint32_t *u_out,
                            const SortPayload *pl, int npl, uint32_t *perm_out, bool counted = false)
{
    int wpb, unit, nblk;
    sort_geometry(N, nbins, wpb, unit, nblk);
    const int64_t ncounts = (int64_t)nbins * nblk;
    const int ntiles = (int)((ncounts + SCAN_TILE - 1) / SCAN_TILE);
    unsigned int *tables = count_tables(ctx, ncounts);
    unsigned int *tiles = (unsigned int *)kde_ws(ctx, WS_SORT_STARTS, (size_t)ntiles * 4);
    if (!tables || !tiles) return KDE_ENOMEM;
    // a counted sort reads the table the gather filled and zeroes the other for the next
    // step; an uncounted one counts into the first table and zeroes the second.
    // count_flip names the table the next counted sort reads (false: first, true: second)
    unsigned int *const t0 = tables, *const t1 = tables + ncounts;
    unsigned int *counts, *other;
    if (counted) {
        counts = ctx->count_flip ? t1 : t0;
        other = ctx->count_flip ? t0 : t1;
        ctx->count_flip = !ctx->count_flip;
    } else {
        counts = t0;
        other = t1;
        ctx->count_flip = true;  // the gather that follows adds into the second table
    }
    const size_t smem = (size_t)wpb * nbins * 4 + (size_t)ntiles * 4;
    static bool attr_set = false;
    if (!attr_set) {
        KDE_CUDA(ctx,
                 cudaFuncSetAttribute(sort_count_kernel<DIGIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024),
                 "sort attribute");
        attr_set = true;
    }
    if (smem > 100 * 1024) return kde_fail(ctx, KDE_ENOTSUP, "sort: %d tiles of counts exceed shared memory", ntiles);
    KdeProfScope _ps(ctx, PROF_SORT);  // the whole pass: count, scan and scatter
    if (!counted) {
        sort_count_kernel<DIGIT><<<nblk, wpb * 32, (size_t)nbins * 4, ctx->stream>>>(u, N, nbins, shift, unit, nblk,
                                                                                    counts);
        KDE_LAUNCHED(ctx, "sort_count_kernel");
    }
    KDE_CUDA(ctx, kde_launch(ctx, true, sort_scan_kernel, dim3(ntiles), dim3(SCAN_THREADS), 0, counts, ncounts, tiles,
                             DIGIT ? nullptr : other),
             "sort_scan_kernel");
    KDE_LAUNCHED(ctx, "sort_scan_kernel");
    ScatterPl sp{};
    sp.n = npl;
    bool narrow = true;
    for (int k = 0; k < npl; ++k) {
        sp.src[k] = pl[k].src;
        sp.dst[k] = pl[k].dst;
        sp.elem[k] = pl[k].elem;
        narrow = narrow && pl[k].elem == 4;
    }
    cudaError_t le;
#define KDE_SCATTER(NPL_, NARROW_)                                                                                  \
    scatter_launch<DIGIT, NPL_, NARROW_>(ctx, nblk, wpb * 32, smem, u, N, nbins, shift, unit, counts, tiles, ntiles, \
                                         u_out, sp, perm_out)
    if constexpr (DIGIT) le = KDE_SCATTER(0, true);
    else if (npl == 0) le = KDE_SCATTER(0, true);
    else if (narrow) {
        switch (npl) {
        case 1: le = KDE_SCATTER(1, true); break;
        case 2: le = KDE_SCATTER(2, true); break;
        case 3: le = KDE_SCATTER(3, true); break;
        default: le = KDE_SCATTER(4, true); break;
        }
    } else {
        switch (npl) {
        case 1: le = KDE_SCATTER(1, false); break;
        case 2: le = KDE_SCATTER(2, false); break;
        case 3: le = KDE_SCATTER(3, false); break;
        default: le = KDE_SCATTER(4, false); break;
        }
    }
#undef KDE_SCATTER
    KDE_CUDA(ctx, le, "sort_scatter_kernel");
    KDE_LAUNCHED(ctx, "sort_scatter_kernel");
    return KDE_OK;
}

kde_status kde_sort_by_bin(kde_ctx *ctx, const uint32_t *u, int64_t N, int nbins, uint32_t *u_out,
                           const SortPayload *pl, int npl, uint32_t *perm_out, bool counted)
{
    if (N <= 0) return KDE_OK;
    if (nbins < 1 || nbins > 8192 || npl > 4 || N > 0xFFFFFFFFll)
        return kde_fail(ctx, KDE_EINVAL, "sort: unsupported sizes");
    return sort_pass<false>(ctx, u, N, nbins, 0, u_out, pl, npl, perm_out, counted);
}

kde_status kde_radix_sort_u32(kde_ctx *ctx, const uint32_t *u, int64_t N, uint32_t *out, uint32_t *tmp)
{
    if (N <= 0) return KDE_OK;
    if (N > 0xFFFFFFFFll) return kde_fail(ctx, KDE_EINVAL, "radix sort: at most 2^32 - 1 keys");
    // LSD: digits 0..3 of 8 bits, u -> tmp -> out -> tmp -> out
    const uint32_t *src = u;
    uint32_t *dst[4] = {tmp, out, tmp, out};
    for (int d = 0; d < 4; ++d) {
        KDE_TRY(sort_pass<true>(ctx, src, N, 256, 8 * d, dst[d], nullptr, 0, nullptr));
        src = dst[d];
    }
    return KDE_OK;
}
