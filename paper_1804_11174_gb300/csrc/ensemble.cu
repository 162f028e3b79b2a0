// ensemble.cu -- many independent PIC realisations advanced together (the
// ensembles behind the MISE and damping-rate statistics of Sec. III).
//
// Realisations are dealt round-robin to `lanes`.  A lane owns a context (its
// own workspace) and a CUDA stream and advances its realisations one after
// another with pic_step, so the lanes run concurrently on the device and small
// realisations no longer leave it idle.  One step of the whole ensemble -- a
// fork from the ensemble's stream to the lanes, every realisation's step, a
// join, and the recording of the step's field energies at a device step
// counter -- is captured once into a CUDA graph and replayed once per step.
// Every realisation runs exactly the kernels pic_step runs on its own state,
// so its results are bitwise those of pic_step alone.
#include "common.cuh"

#define ENS_MAX_LANES 16

struct kde_ensemble {
    kde_ctx *ctx = nullptr;  // the caller's context: its stream orders the calls
    int R = 0, nl = 0;
    double L = 0, dt = 0;
    std::vector<pic_state> ps;
    std::vector<int64_t> off;
    std::vector<int> goff;
    std::vector<kde_ctx *> lane_ctx;
    std::vector<cudaStream_t> lane_st;
    std::vector<cudaEvent_t> lane_ev;
    cudaEvent_t fork_ev = nullptr;
    cudaStream_t stream = nullptr;  // the ensemble's own stream (graph capture and replay)
    double *W = nullptr;            // device float64[R]: field energy of the step just run
    int *d_step = nullptr;          // device: step index inside the current run
    float *rho = nullptr;           // device float32[sum Ng]: densities for the MISE
    int2 *d_grid = nullptr;         // device (first node, Ng) per realisation
    int64_t steps_done = 0;
    cudaGraphExec_t graph = nullptr;
    double *graph_energy = nullptr;
    int graph_nmax = -1;
};

__global__ void ens_record_kernel(const double *W, int R, double *energy, int nmax, const int *step)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = *step;
    if (r < R && energy && k >= 0 && k < nmax) energy[(size_t)r * nmax + k] = W[r];
}

__global__ void ens_advance_kernel(int *step) { *step += 1; }

// dx sum_g (rho_g - (1 + alpha cos(2 pi mode g / Ng)))^2 per realisation, FP64
__global__ void ens_mise_kernel(const float *rho, const int2 *grid, double L, double alpha, int mode, double *mise)
{
    __shared__ double red[256];
    const int2 gd = grid[blockIdx.x];
    double s = 0.0;
    for (int g = threadIdx.x; g < gd.y; g += 256) {
        const double d = (double)rho[gd.x + g] - (1.0 + alpha * cospi(2.0 * mode * (double)g / gd.y));
        s += d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) mise[blockIdx.x] = red[0] * (L / gd.y);
}

// fork the lanes off the ensemble's stream
static kde_status ens_fork(kde_ensemble *e)
{
    KDE_CUDA(e->ctx, cudaEventRecord(e->fork_ev, e->stream), "ensemble fork");
    for (int l = 0; l < e->nl; ++l)
        KDE_CUDA(e->ctx, cudaStreamWaitEvent(e->lane_st[l], e->fork_ev, 0), "ensemble fork wait");
    return KDE_OK;
}

// join the lanes back into the ensemble's stream
static kde_status ens_join(kde_ensemble *e)
{
    for (int l = 0; l < e->nl; ++l) {
        KDE_CUDA(e->ctx, cudaEventRecord(e->lane_ev[l], e->lane_st[l]), "ensemble join");
        KDE_CUDA(e->ctx, cudaStreamWaitEvent(e->stream, e->lane_ev[l], 0), "ensemble join wait");
    }
    return KDE_OK;
}

// one step of every realisation plus the energy record (on the ensemble's stream)
static kde_status ens_enqueue_step(kde_ensemble *e, double *energy, int nmax, bool first)
{
    KDE_TRY(ens_fork(e));
    for (int r = 0; r < e->R; ++r) {
        pic_state &s = e->ps[r];
        kde_ctx *lc = e->lane_ctx[r % e->nl];
        s.step = 0;  // energy slot W[r]; the kick is set by the flag
        s.flags = first ? 0u : PIC_NO_BACKSTEP;
        if (first) {
            // one autotuner table for the whole ensemble: a key tuned on one lane is reused
            // by the others (the host issues the realisations in order, and tuning waits
            // for its own runs); the caller's context keeps the union
            lc->gat2_tuned.insert(e->ctx->gat2_tuned.begin(), e->ctx->gat2_tuned.end());
            lc->cut_tuned.insert(e->ctx->cut_tuned.begin(), e->ctx->cut_tuned.end());
        }
        kde_status st = pic_step(lc, &s, 1);
        s.step = 0;
        if (st != KDE_OK) return kde_fail(e->ctx, st, "ensemble realisation %d: %s", r, kde_last_error(lc));
        if (first) {
            e->ctx->gat2_tuned.insert(lc->gat2_tuned.begin(), lc->gat2_tuned.end());
            e->ctx->cut_tuned.insert(lc->cut_tuned.begin(), lc->cut_tuned.end());
        }
    }
    KDE_TRY(ens_join(e));
    ens_record_kernel<<<(e->R + 255) / 256, 256, 0, e->stream>>>(e->W, e->R, energy, nmax, e->d_step);
    KDE_LAUNCHED(e->ctx, "ens_record_kernel");
    ens_advance_kernel<<<1, 1, 0, e->stream>>>(e->d_step);
    KDE_LAUNCHED(e->ctx, "ens_advance_kernel");
    return KDE_OK;
}

extern "C" kde_status kde_ensemble_destroy(kde_ensemble *e);

extern "C" kde_status kde_ensemble_create(kde_ctx *ctx, kde_ensemble **out, int32_t R, const int64_t *N_host,
                                          const int32_t *Ng_host, const double *kappa_host, double L, double dt,
                                          uint32_t *u, float *v)
{
    if (!ctx) return KDE_EINVAL;
    if (!out || R < 1 || !N_host || !Ng_host || !kappa_host || !(L > 0) || !(dt > 0) || !u || !v)
        return kde_fail(ctx, KDE_EINVAL, "kde_ensemble_create: bad arguments");
    *out = nullptr;
    int64_t off = 0;
    int goff = 0;
    for (int r = 0; r < R; ++r) {
        if (N_host[r] < 1 || N_host[r] > 0xFFFFFFFFll || Ng_host[r] < 1 || Ng_host[r] > KDE_MAX_NG ||
            !(kappa_host[r] > 0 && kappa_host[r] <= KDE_KAPPA_MAX))
            return kde_fail(ctx, KDE_EINVAL, "kde_ensemble_create: realisation %d needs 1 <= N < 2^32, "
                            "1 <= Ng <= %d and a width in (0, 1e6]", r, KDE_MAX_NG);
        off += N_host[r];
        goff += Ng_host[r];
    }
    cudaSetDevice(ctx->device);
    kde_ensemble *e = new kde_ensemble();
    e->ctx = ctx;
    e->R = R;
    e->L = L;
    e->dt = dt;
    e->nl = R < ENS_MAX_LANES ? R : ENS_MAX_LANES;
    cudaError_t err = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->fork_ev, cudaEventDisableTiming);
    for (int l = 0; err == cudaSuccess && l < e->nl; ++l) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        err = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (err == cudaSuccess) e->lane_st.push_back(st);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (err == cudaSuccess) e->lane_ev.push_back(ev);
        kde_ctx *lc = nullptr;
        if (err == cudaSuccess && kde_create(&lc, ctx->device, st) != KDE_OK) err = cudaErrorMemoryAllocation;
        if (err == cudaSuccess) {
            lc->autotune = ctx->autotune;  // lanes tune in the uncaptured first step
            lc->cut_fixed = ctx->cut_fixed;
            lc->overlap = ctx->overlap;
            e->lane_ctx.push_back(lc);
        }
    }
    if (err == cudaSuccess) err = cudaMalloc(&e->W, sizeof(double) * R);
    if (err == cudaSuccess) err = cudaMalloc(&e->d_step, sizeof(int));
    if (err == cudaSuccess) err = cudaMalloc(&e->rho, sizeof(float) * (size_t)goff);
    if (err == cudaSuccess) err = cudaMalloc(&e->d_grid, sizeof(int2) * R);
    std::vector<int2> grid(R);
    off = 0;
    goff = 0;
    for (int r = 0; r < R; ++r) {
        pic_state s{};
        s.u = u + off;
        s.v = v + off;
        s.N = N_host[r];
        s.Ng = Ng_host[r];
        s.L = L;
        s.dt = dt;
        s.qm = -1.0;
        s.charge = -1.0;
        s.background = 1.0;
        s.kappa_uniform = kappa_host[r];
        s.energy = e->W + r;
        e->ps.push_back(s);
        e->off.push_back(off);
        e->goff.push_back(goff);
        grid[r] = make_int2(goff, Ng_host[r]);
        off += N_host[r];
        goff += Ng_host[r];
    }
    if (err == cudaSuccess)
        err = cudaMemcpy(e->d_grid, grid.data(), sizeof(int2) * R, cudaMemcpyHostToDevice);
    if (err != cudaSuccess) {
        cudaGetLastError();
        kde_ensemble_destroy(e);
        return kde_fail(ctx, KDE_ENOMEM, "kde_ensemble_create: allocation failed");
    }
    *out = e;
    return KDE_OK;
}

extern "C" kde_status kde_ensemble_set_widths(kde_ensemble *e, const double *kappa_host)
{
    if (!e || !kappa_host) return KDE_EINVAL;
    for (int r = 0; r < e->R; ++r)
        if (!(kappa_host[r] > 0 && kappa_host[r] <= KDE_KAPPA_MAX))
            return kde_fail(e->ctx, KDE_EINVAL, "kde_ensemble_set_widths: width %d outside (0, 1e6]", r);
    for (int r = 0; r < e->R; ++r) e->ps[r].kappa_uniform = kappa_host[r];
    // the widths are launch parameters baked into a captured step: capture again
    if (e->graph) {
        cudaSetDevice(e->ctx->device);
        cudaStreamSynchronize(e->stream);
        cudaGraphExecDestroy(e->graph);
        e->graph = nullptr;
    }
    return KDE_OK;
}

extern "C" kde_status kde_ensemble_set_shape(kde_ensemble *e, int32_t order, double h)
{
    if (!e) return KDE_EINVAL;
    if (!(order == 0 || order == 1 || order == 2 || order == 3 || order == 5) || h < 0)
        return kde_fail(e->ctx, KDE_EINVAL, "kde_ensemble_set_shape: order in {0, 1, 2, 3, 5}, h >= 0");
    for (int r = 0; r < e->R; ++r) {
        e->ps[r].shape_order = order;
        e->ps[r].shape_h = h;
    }
    if (e->graph) {
        cudaSetDevice(e->ctx->device);
        cudaStreamSynchronize(e->stream);
        cudaGraphExecDestroy(e->graph);
        e->graph = nullptr;
    }
    return KDE_OK;
}

extern "C" kde_status kde_ensemble_mise(kde_ensemble *e, double alpha, int32_t mode, double *mise)
{
    if (!e || !mise) return KDE_EINVAL;
    kde_ctx *ctx = e->ctx;
    cudaSetDevice(ctx->device);
    cudaEvent_t ev;
    KDE_CUDA(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "ensemble event");
    cudaEventRecord(ev, ctx->stream);
    cudaStreamWaitEvent(e->stream, ev, 0);
    kde_status s = ens_fork(e);
    for (int r = 0; s == KDE_OK && r < e->R; ++r) {
        const pic_state &p = e->ps[r];
        kde_ctx *lc = e->lane_ctx[r % e->nl];
        s = kde_deposit(lc, p.u, nullptr, p.kappa_uniform, nullptr, p.N, p.Ng, e->L, e->rho + e->goff[r], 0);
        if (s != KDE_OK) s = kde_fail(ctx, s, "ensemble MISE deposit %d: %s", r, kde_last_error(lc));
    }
    if (s == KDE_OK) s = ens_join(e);
    if (s == KDE_OK) {
        ens_mise_kernel<<<e->R, 256, 0, e->stream>>>(e->rho, e->d_grid, e->L, alpha, mode, mise);
        s = kde_cuda_check(ctx, cudaGetLastError(), "ens_mise_kernel");
        ++ctx->launches;
    }
    cudaEventRecord(ev, e->stream);
    cudaStreamWaitEvent(ctx->stream, ev, 0);
    cudaEventDestroy(ev);
    return s;
}

extern "C" kde_status kde_ensemble_run(kde_ensemble *e, int32_t n_steps, double *energy, int32_t use_graph)
{
    if (!e || n_steps < 0) return KDE_EINVAL;
    kde_ctx *ctx = e->ctx;
    cudaSetDevice(ctx->device);
    cudaEvent_t ev;
    KDE_CUDA(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "ensemble event");
    cudaEventRecord(ev, ctx->stream);
    cudaStreamWaitEvent(e->stream, ev, 0);
    kde_status s = kde_cuda_check(ctx, cudaMemsetAsync(e->d_step, 0, sizeof(int), e->stream), "step reset");
    int k = 0;
    // the first step of the ensemble's life carries the half kick; it also sizes every
    // lane's workspace and tables, so that a captured step allocates nothing
    if (s == KDE_OK && k < n_steps && e->steps_done == 0) {
        s = ens_enqueue_step(e, energy, n_steps, true);
        ++k;
        ++e->steps_done;
    }
    if (s == KDE_OK && k < n_steps && use_graph) {
        if (!e->graph || e->graph_energy != energy || e->graph_nmax != n_steps) {
            if (e->graph) {
                cudaStreamSynchronize(e->stream);
                cudaGraphExecDestroy(e->graph);
                e->graph = nullptr;
            }
            std::vector<bool> prof(e->nl);
            for (int l = 0; l < e->nl; ++l) {
                prof[l] = e->lane_ctx[l]->prof_on;
                e->lane_ctx[l]->prof_on = false;  // no event records inside the captured step
            }
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                s = kde_fail(ctx, KDE_ECUDA, "ensemble graph capture could not start");
            if (s == KDE_OK) s = ens_enqueue_step(e, energy, n_steps, false);
            const cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
            for (int l = 0; l < e->nl; ++l) e->lane_ctx[l]->prof_on = prof[l];
            if (s == KDE_OK && ce != cudaSuccess) s = kde_cuda_check(ctx, ce, "ensemble graph capture");
            if (s == KDE_OK && cudaGraphInstantiate(&e->graph, g, 0) != cudaSuccess)
                s = kde_fail(ctx, KDE_ECUDA, "ensemble graph instantiation failed");
            if (g) cudaGraphDestroy(g);
            if (s != KDE_OK) cudaGetLastError();
            e->graph_energy = energy;
            e->graph_nmax = n_steps;
        }
        for (; s == KDE_OK && k < n_steps; ++k) {
            if (cudaGraphLaunch(e->graph, e->stream) != cudaSuccess) s = kde_fail(ctx, KDE_ECUDA, "graph launch failed");
            ++e->steps_done;
        }
    }
    for (; s == KDE_OK && k < n_steps; ++k) {
        s = ens_enqueue_step(e, energy, n_steps, false);
        ++e->steps_done;
    }
    cudaEventRecord(ev, e->stream);
    cudaStreamWaitEvent(ctx->stream, ev, 0);
    cudaEventDestroy(ev);
    return s;
}

extern "C" kde_status kde_ensemble_destroy(kde_ensemble *e)
{
    if (!e) return KDE_EINVAL;
    cudaSetDevice(e->ctx->device);
    if (e->stream) cudaStreamSynchronize(e->stream);
    for (auto st : e->lane_st) cudaStreamSynchronize(st);
    if (e->graph) cudaGraphExecDestroy(e->graph);
    for (auto *lc : e->lane_ctx) kde_destroy(lc);
    for (auto st : e->lane_st) cudaStreamDestroy(st);
    for (auto ev : e->lane_ev) cudaEventDestroy(ev);
    if (e->fork_ev) cudaEventDestroy(e->fork_ev);
    void *ps[] = {e->W, e->d_step, e->rho, e->d_grid};
    for (void *p : ps)
        if (p) cudaFree(p);
    if (e->stream) cudaStreamDestroy(e->stream);
    delete e;
    return KDE_OK;
}
