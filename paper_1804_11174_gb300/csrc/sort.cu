// sort.cu -- stable counting sort of particles by bin (cell) index.
//
// Each warp owns a contiguous unit of `unit` particles (a multiple of 32).
//   count   : warp-private shared histogram of its unit -> counts[bin][unit]
//             (bin-major, so that the destination order of the segments is the
//             flat index bin * nunits + unit)
//   scan    : exclusive scan of the flat counts array: tiles of 4096 scanned
//             in place plus a one-block scan of the tile totals
//   scatter : the warp loads its unit up front, then ranks equal keys in each
//             32-particle step with __match_any_sync and writes every particle
//             (position and payloads) to its segment start + running count +
//             rank.
// The order inside a bin is the input order (stable), so results are
// deterministic.  Units are small enough to keep thousands of warps in flight.
//
// The same kernels in digit mode (key = a bit field of the code) give an LSD
// radix sort of the full 32-bit codes: four stable passes of 8-bit digits.
#include "common.cuh"

#define SORT_MAX_COUNTS (1 << 22)
#define SCAN_TILE 4096
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

template <bool DIGIT>
__global__ void sort_count_kernel(const uint32_t *__restrict__ u, int64_t N, int nbins, int shift, int unit,
                                  int nunits, unsigned int *counts)
{
    extern __shared__ unsigned int hist[];
    const int wpb = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int un = blockIdx.x * wpb + warp;
    unsigned int *h = hist + (size_t)warp * nbins;
    for (int b = lane; b < nbins; b += 32) h[b] = 0;
    __syncwarp();
    if (un >= nunits) return;
    const int64_t i0 = (int64_t)un * unit, i1 = i0 + unit < N ? i0 + unit : N;
    for (int64_t i = i0 + lane; i < i1; i += 32) atomicAdd(&h[sort_key<DIGIT>(u[i], nbins, shift)], 1u);
    __syncwarp();
    for (int b = lane; b < nbins; b += 32) counts[(size_t)b * nunits + un] = h[b];
}

// exclusive scan of each SCAN_TILE-element tile in place; tile totals out
__global__ void __launch_bounds__(SCAN_THREADS) sort_scan_tiles_kernel(unsigned int *a, int64_t n, unsigned int *tot)
{
    __shared__ unsigned int wsum[SCAN_THREADS / 32];
    const int per = SCAN_TILE / SCAN_THREADS;  // 16 consecutive elements per thread
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * per;
    unsigned int v[SCAN_TILE / SCAN_THREADS];
    unsigned int s = 0;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        v[k] = base + k < n ? a[base + k] : 0u;
        s += v[k];
    }
    // exclusive scan of the per-thread sums across the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned int inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    unsigned int woff = 0, total = 0;
    for (int w = 0; w < SCAN_THREADS / 32; ++w) {
        if (w < warp) woff += wsum[w];
        total += wsum[w];
    }
    unsigned int run = woff + inc - s;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        if (base + k < n) a[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) tot[blockIdx.x] = total;
}

// exclusive scan of the tile totals (at most 1024) in one block
__global__ void sort_scan_totals_kernel(unsigned int *tot, int ntiles)
{
    __shared__ unsigned int wsum[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    unsigned int v = t < ntiles ? tot[t] : 0u;
    unsigned int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned int x = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += x;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    unsigned int woff = 0;
    for (int w = 0; w < warp; ++w) woff += wsum[w];
    if (t < ntiles) tot[t] = woff + inc - v;
}

struct ScatterPl {
    const void *src[4];
    void *dst[4];
    int elem[4];
    int n;
};

#define SORT_MAXR 8  // 32-particle steps loaded ahead per chunk of the unit

template <bool DIGIT>
__global__ void sort_scatter_kernel(const uint32_t *__restrict__ u, int64_t N, int nbins, int shift, int unit,
                                    int nunits, const unsigned int *__restrict__ seg,
                                    const unsigned int *__restrict__ tiles, uint32_t *u_out, ScatterPl pl,
                                    uint32_t *perm_out)
{
    extern __shared__ unsigned int hist[];
    const int wpb = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int un = blockIdx.x * wpb + warp;
    unsigned int *h = hist + (size_t)warp * nbins;
    if (un >= nunits) return;
    for (int b = lane; b < nbins; b += 32) h[b] = 0;
    __syncwarp();
    const unsigned int lt = (1u << lane) - 1u;
    const int64_t i0 = (int64_t)un * unit, i1 = i0 + unit < N ? i0 + unit : N;
    for (int64_t c0 = i0; c0 < i1; c0 += 32 * SORT_MAXR) {
        uint32_t uu[SORT_MAXR];
#pragma unroll
        for (int r = 0; r < SORT_MAXR; ++r) {
            const int64_t i = c0 + r * 32 + lane;
            uu[r] = i < i1 ? u[i] : 0u;
        }
#pragma unroll
        for (int r = 0; r < SORT_MAXR; ++r) {
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
            if (valid) {
                const size_t flat = (size_t)key * nunits + un;
                const size_t dst = (size_t)seg[flat] + tiles[flat / SCAN_TILE] + before + rank;
                u_out[dst] = uu[r];
                for (int k = 0; k < pl.n; ++k) {
                    if (pl.elem[k] == 8) ((uint64_t *)pl.dst[k])[dst] = ((const uint64_t *)pl.src[k])[i];
                    else ((uint32_t *)pl.dst[k])[dst] = ((const uint32_t *)pl.src[k])[i];
                }
                if (perm_out) perm_out[dst] = (uint32_t)i;
            }
        }
    }
}

template <bool DIGIT>
static kde_status sort_pass(kde_ctx *ctx, const uint32_t *u, int64_t N, int nbins, int shift, uint32_t *u_out,
                            const SortPayload *pl, int npl, uint32_t *perm_out)
{
    int unit = 256;
    while ((int64_t)nbins * ((N + unit - 1) / unit) > SORT_MAX_COUNTS) unit *= 2;
    const int nunits = (int)((N + unit - 1) / unit);
    const int64_t ncounts = (int64_t)nbins * nunits;
    const int ntiles = (int)((ncounts + SCAN_TILE - 1) / SCAN_TILE);
    unsigned int *counts = (unsigned int *)kde_ws(ctx, WS_SORT_COUNTS, (size_t)ncounts * 4);
    unsigned int *tiles = (unsigned int *)kde_ws(ctx, WS_SORT_STARTS, (size_t)ntiles * 4);
    if (!counts || !tiles) return KDE_ENOMEM;
    // warps per block: warp-private histograms must fit the shared-memory budget
    int wpb = 8;
    while (wpb > 1 && (size_t)wpb * nbins * 4 > 96 * 1024) wpb >>= 1;
    const size_t smem = (size_t)wpb * nbins * 4;
    static bool attr_set = false;
    if (!attr_set) {
        KDE_CUDA(ctx,
                 cudaFuncSetAttribute(sort_count_kernel<DIGIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024),
                 "sort attribute");
        KDE_CUDA(ctx,
                 cudaFuncSetAttribute(sort_scatter_kernel<DIGIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      96 * 1024),
                 "sort attribute");
        attr_set = true;
    }
    const int blocks = (nunits + wpb - 1) / wpb;
    sort_count_kernel<DIGIT><<<blocks, wpb * 32, smem, ctx->stream>>>(u, N, nbins, shift, unit, nunits, counts);
    KDE_LAUNCHED(ctx, "sort_count_kernel");
    sort_scan_tiles_kernel<<<ntiles, SCAN_THREADS, 0, ctx->stream>>>(counts, ncounts, tiles);
    KDE_LAUNCHED(ctx, "sort_scan_tiles_kernel");
    sort_scan_totals_kernel<<<1, 1024, 0, ctx->stream>>>(tiles, ntiles);
    KDE_LAUNCHED(ctx, "sort_scan_totals_kernel");
    ScatterPl sp{};
    sp.n = npl;
    for (int k = 0; k < npl; ++k) {
        sp.src[k] = pl[k].src;
        sp.dst[k] = pl[k].dst;
        sp.elem[k] = pl[k].elem;
    }
    {
        KdeProfScope _ps(ctx, PROF_SORT);
        sort_scatter_kernel<DIGIT><<<blocks, wpb * 32, smem, ctx->stream>>>(u, N, nbins, shift, unit, nunits, counts,
                                                                            tiles, u_out, sp, perm_out);
    }
    KDE_LAUNCHED(ctx, "sort_scatter_kernel");
    return KDE_OK;
}

kde_status kde_sort_by_bin(kde_ctx *ctx, const uint32_t *u, int64_t N, int nbins, uint32_t *u_out,
                           const SortPayload *pl, int npl, uint32_t *perm_out)
{
    if (N <= 0) return KDE_OK;
    if (nbins < 1 || nbins > 8192 || npl > 4 || N > 0xFFFFFFFFll)
        return kde_fail(ctx, KDE_EINVAL, "sort: unsupported sizes");
    return sort_pass<false>(ctx, u, N, nbins, 0, u_out, pl, npl, perm_out);
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
