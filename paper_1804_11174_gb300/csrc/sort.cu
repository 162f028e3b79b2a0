// sort.cu -- stable counting sort of particles by bin (cell) index.
//
// Three passes, each warp owning a contiguous unit of SORT_UNIT particles:
//   count   : warp-private shared histogram of its unit -> counts[unit][bin]
//   scan    : per bin, exclusive prefix over units; then exclusive prefix of
//             the bin totals -> bin starts
//   scatter : the warp re-reads its unit in order, ranks equal keys within
//             each 32-particle step with __match_any_sync, and writes every
//             particle (position + payloads) to
//             start[bin] + prefix[unit][bin] + running count + rank.
// The order inside a bin is the input order (stable), so the result is
// deterministic.
#include "common.cuh"

#define SORT_UNIT 4096
#define SORT_WARPS 4

__device__ __forceinline__ int bin_of(uint32_t u, int nbins) { return (int)(((uint64_t)u * (uint64_t)nbins) >> 32); }

__global__ void __launch_bounds__(SORT_WARPS * 32) sort_count_kernel(const uint32_t *u, int64_t N, int nbins,
                                                                      int nunits, unsigned int *counts)
{
    extern __shared__ unsigned int hist[];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int unit = blockIdx.x * SORT_WARPS + warp;
    unsigned int *h = hist + (size_t)warp * nbins;
    for (int b = lane; b < nbins; b += 32) h[b] = 0;
    __syncwarp();
    if (unit < nunits) {
        int64_t i0 = (int64_t)unit * SORT_UNIT, i1 = i0 + SORT_UNIT < N ? i0 + SORT_UNIT : N;
        for (int64_t i = i0 + lane; i < i1; i += 32) atomicAdd(&h[bin_of(u[i], nbins)], 1u);
        __syncwarp();
        for (int b = lane; b < nbins; b += 32) counts[(size_t)unit * nbins + b] = h[b];
    }
}

// counts[unit][bin] -> exclusive prefix over units (in place); totals[bin]
__global__ void sort_colscan_kernel(unsigned int *counts, int nbins, int nunits, unsigned int *totals)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    unsigned int run = 0;
    for (int t = 0; t < nunits; ++t) {
        unsigned int c = counts[(size_t)t * nbins + b];
        counts[(size_t)t * nbins + b] = run;
        run += c;
    }
    totals[b] = run;
}

// exclusive scan of totals[nbins] in one block (in place)
__global__ void sort_binscan_kernel(unsigned int *totals, int nbins)
{
    __shared__ unsigned int part[1024];
    int t = threadIdx.x, per = (nbins + blockDim.x - 1) / blockDim.x;
    int b0 = t * per, b1 = b0 + per < nbins ? b0 + per : nbins;
    unsigned int s = 0;
    for (int b = b0; b < b1; ++b) s += totals[b];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        unsigned int run = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) {
            unsigned int c = part[k];
            part[k] = run;
            run += c;
        }
    }
    __syncthreads();
    unsigned int run = part[t];
    for (int b = b0; b < b1; ++b) {
        unsigned int c = totals[b];
        totals[b] = run;
        run += c;
    }
}

struct ScatterPl {
    const void *src[4];
    void *dst[4];
    int elem[4];
    int n;
};

__global__ void __launch_bounds__(SORT_WARPS * 32)
    sort_scatter_kernel(const uint32_t *u, int64_t N, int nbins, int nunits, const unsigned int *prefix,
                        const unsigned int *starts, uint32_t *u_out, ScatterPl pl, uint32_t *perm_out)
{
    extern __shared__ unsigned int hist[];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int unit = blockIdx.x * SORT_WARPS + warp;
    unsigned int *h = hist + (size_t)warp * nbins;
    if (unit >= nunits) return;
    for (int b = lane; b < nbins; b += 32) h[b] = 0;
    __syncwarp();
    const unsigned int *pre = prefix + (size_t)unit * nbins;
    unsigned int lt = (1u << lane) - 1u;
    int64_t i0 = (int64_t)unit * SORT_UNIT, i1 = i0 + SORT_UNIT < N ? i0 + SORT_UNIT : N;
    for (int64_t base = i0; base < i1; base += 32) {
        int64_t i = base + lane;
        bool valid = i < i1;
        uint32_t uu = valid ? u[i] : 0u;
        int key = valid ? bin_of(uu, nbins) : -1;
        unsigned int peers = __match_any_sync(0xffffffffu, key);
        unsigned int rank = __popc(peers & lt);
        unsigned int before = valid ? h[key] : 0u;
        __syncwarp();
        if (valid && rank == 0) h[key] = before + __popc(peers);
        __syncwarp();
        if (valid) {
            size_t dst = (size_t)starts[key] + pre[key] + before + rank;
            u_out[dst] = uu;
            for (int k = 0; k < pl.n; ++k) {
                if (pl.elem[k] == 8) ((uint64_t *)pl.dst[k])[dst] = ((const uint64_t *)pl.src[k])[i];
                else ((uint32_t *)pl.dst[k])[dst] = ((const uint32_t *)pl.src[k])[i];
            }
            if (perm_out) perm_out[dst] = (uint32_t)i;
        }
    }
}

kde_status kde_sort_by_bin(kde_ctx *ctx, const uint32_t *u, int64_t N, int nbins, uint32_t *u_out,
                           const SortPayload *pl, int npl, uint32_t *perm_out)
{
    if (N <= 0) return KDE_OK;
    if (nbins < 1 || nbins > 8192 || npl > 4 || N > 0xFFFFFFFFll)
        return kde_fail(ctx, KDE_EINVAL, "sort: unsupported sizes");
    int nunits = (int)((N + SORT_UNIT - 1) / SORT_UNIT);
    unsigned int *counts = (unsigned int *)kde_ws(ctx, WS_SORT_COUNTS, (size_t)nunits * nbins * 4);
    unsigned int *starts = (unsigned int *)kde_ws(ctx, WS_SORT_STARTS, (size_t)nbins * 4);
    if (!counts || !starts) return KDE_ENOMEM;
    size_t smem = (size_t)SORT_WARPS * nbins * 4;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(sort_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SORT_WARPS * 8192 * 4);
        cudaFuncSetAttribute(sort_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SORT_WARPS * 8192 * 4);
        attr_set = true;
    }
    int blocks = (nunits + SORT_WARPS - 1) / SORT_WARPS;
    sort_count_kernel<<<blocks, SORT_WARPS * 32, smem, ctx->stream>>>(u, N, nbins, nunits, counts);
    KDE_LAUNCHED(ctx, "sort_count_kernel");
    sort_colscan_kernel<<<(nbins + 127) / 128, 128, 0, ctx->stream>>>(counts, nbins, nunits, starts);
    KDE_LAUNCHED(ctx, "sort_colscan_kernel");
    sort_binscan_kernel<<<1, 1024, 0, ctx->stream>>>(starts, nbins);
    KDE_LAUNCHED(ctx, "sort_binscan_kernel");
    ScatterPl sp{};
    sp.n = npl;
    for (int k = 0; k < npl; ++k) {
        sp.src[k] = pl[k].src;
        sp.dst[k] = pl[k].dst;
        sp.elem[k] = pl[k].elem;
    }
    {
        KdeProfScope _ps(ctx, PROF_SORT);
    sort_scatter_kernel<<<blocks, SORT_WARPS * 32, smem, ctx->stream>>>(u, N, nbins, nunits, counts, starts, u_out,
                                                                         sp, perm_out);
    }
    KDE_LAUNCHED(ctx, "sort_scatter_kernel");
    return KDE_OK;
}
