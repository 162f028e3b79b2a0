// server.cu -- request server for the KDE-PIC operations (deposit, gather,
// CV, short PIC runs) with continuous batching.
//
// Each of `n_slots` slots owns a context (its own workspace) and a CUDA stream
// and runs on its own host thread.  Submitted requests wait in one FIFO queue;
// the head request is admitted as soon as a slot is idle and its device
// footprint fits in what the HBM budget has left, so requests that arrive
// while others run start as slots and memory free up and their kernels overlap
// on the device.  Per request the slot allocates its device buffers from the
// stream-ordered pool (cudaMallocAsync), copies the host inputs, runs the
// library's entry points on its stream, copies the results back and frees the
// buffers; the caller's host buffers are read and written only by that slot.
// Because every kernel is deterministic and a request only touches its own
// buffers and its slot's workspace, a result does not depend on which other
// requests ran beside it.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "common.cuh"

namespace {

using clk = std::chrono::steady_clock;

struct Ticket {
    kde_request req;
    clk::time_point t_submit, t_start, t_end;
    kde_status status = KDE_OK;
    bool done = false;
    int64_t footprint = 0;
    std::string err;
};

}  // namespace

struct kde_server {
    int device = 0;
    int64_t budget = 0, in_use = 0;
    std::vector<std::thread> workers;
    std::vector<kde_ctx *> ctxs;
    std::vector<cudaStream_t> streams;
    std::mutex mu;
    std::condition_variable cv_queue, cv_done;
    std::deque<int64_t> queue;
    std::unordered_map<int64_t, Ticket> tickets;
    int64_t next_id = 1;
    bool stop = false;
    int64_t served = 0;
};

static int64_t request_footprint(const kde_request &r)
{
    // inputs, outputs and the slot workspace a request of this size grows (sort
    // copies, CV tables), in bytes
    const int64_t N = r.N, Ng = r.Ng;
    int64_t b = N * 16 + Ng * 16 + (1 << 20);
    if (r.kind == KDE_REQ_CV) b += N * (8 + 12 + 4 * (int64_t)r.n_cand) + (1 << 22);
    else b += N * 40 + (16 << 20);
    return b;
}

static kde_status run_request(kde_server *S, kde_ctx *ctx, cudaStream_t st, const kde_request &r)
{
    const int64_t N = r.N;
    void *bufs[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    auto dalloc = [&](int slot, size_t bytes) -> void * {
        if (cudaMallocAsync(&bufs[slot], bytes ? bytes : 16, st) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return bufs[slot];
    };
    kde_status rc = KDE_OK;
    uint32_t *du = (uint32_t *)dalloc(0, (size_t)N * 4);
    float *dk = r.kappa ? (float *)dalloc(1, (size_t)N * 4) : nullptr;
    if (!du || (r.kappa && !dk)) rc = KDE_ENOMEM;
    if (rc == KDE_OK && N > 0) {
        cudaMemcpyAsync(du, r.u, (size_t)N * 4, cudaMemcpyHostToDevice, st);
        if (dk) cudaMemcpyAsync(dk, r.kappa, (size_t)N * 4, cudaMemcpyHostToDevice, st);
    }
    if (rc == KDE_OK) {
        switch (r.kind) {
        case KDE_REQ_DEPOSIT: {
            float *drho = (float *)dalloc(2, (size_t)r.Ng * 4);
            if (!drho) {
                rc = KDE_ENOMEM;
                break;
            }
            rc = kde_deposit(ctx, du, dk, r.kappa_uniform, nullptr, N, r.Ng, r.L, drho, 0);
            if (rc == KDE_OK) cudaMemcpyAsync(r.out, drho, (size_t)r.Ng * 4, cudaMemcpyDeviceToHost, st);
            break;
        }
        case KDE_REQ_GATHER: {
            float *df = (float *)dalloc(2, (size_t)r.Ng * 4);
            float *de = (float *)dalloc(3, (size_t)N * 4);
            if (!df || !de) {
                rc = KDE_ENOMEM;
                break;
            }
            cudaMemcpyAsync(df, r.field, (size_t)r.Ng * 4, cudaMemcpyHostToDevice, st);
            rc = kde_gather(ctx, du, dk, r.kappa_uniform, N, df, r.Ng, r.L, de, 0);
            if (rc == KDE_OK) cudaMemcpyAsync(r.out, de, (size_t)N * 4, cudaMemcpyDeviceToHost, st);
            break;
        }
        case KDE_REQ_CV: {
            int32_t am = 0;
            rc = kde_cv(ctx, du, dk, N, r.L, r.cand, r.n_cand, r.out64, &am, nullptr,
                        (dk ? KDE_CV_SCALE : 0) | (r.flags & KDE_CV_SPECTRAL));
            if (rc == KDE_OK && r.out_argmin) *r.out_argmin = am;
            break;
        }
        case KDE_REQ_PIC: {
            float *dv = (float *)dalloc(2, (size_t)N * 4);
            float *dn = dk ? (float *)dalloc(3, (size_t)N * 4) : nullptr;
            double *den = (double *)dalloc(4, (size_t)(r.n_steps > 0 ? r.n_steps : 1) * 8);
            if (!dv || (dk && !dn) || !den) {
                rc = KDE_ENOMEM;
                break;
            }
            cudaMemcpyAsync(dv, r.v, (size_t)N * 4, cudaMemcpyHostToDevice, st);
            pic_state ps{};
            ps.u = du;
            ps.v = dv;
            ps.kappa = dk;
            ps.kappa_norm = dn;
            ps.N = N;
            ps.Ng = r.Ng;
            ps.L = r.L;
            ps.dt = r.dt;
            ps.qm = -1.0;
            ps.charge = -1.0;
            ps.background = 1.0;
            ps.kappa_uniform = r.kappa_uniform;
            ps.energy = den;
            rc = pic_step(ctx, &ps, r.n_steps);
            if (rc == KDE_OK) {
                cudaMemcpyAsync(r.out64, den, (size_t)r.n_steps * 8, cudaMemcpyDeviceToHost, st);
                if (r.out) cudaMemcpyAsync(r.out, dv, (size_t)N * 4, cudaMemcpyDeviceToHost, st);
            }
            break;
        }
        default:
            rc = KDE_EINVAL;
        }
    }
    for (int k = 0; k < 6; ++k)
        if (bufs[k]) cudaFreeAsync(bufs[k], st);
    kde_status s2 = kde_sync(ctx);
    if (rc == KDE_OK) rc = s2;
    (void)S;
    return rc;
}

static void worker_main(kde_server *S, int slot)
{
    cudaSetDevice(S->device);
    kde_ctx *ctx = S->ctxs[slot];
    cudaStream_t st = S->streams[slot];
    for (;;) {
        int64_t id;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            // FIFO admission: the head request starts when its footprint fits the budget
            S->cv_queue.wait(lk, [&] {
                return S->stop ||
                       (!S->queue.empty() &&
                        (S->in_use == 0 || S->in_use + S->tickets[S->queue.front()].footprint <= S->budget));
            });
            if (S->stop && S->queue.empty()) return;
            id = S->queue.front();
            S->queue.pop_front();
            Ticket &t = S->tickets[id];
            S->in_use += t.footprint;
            t.t_start = clk::now();
        }
        kde_request req;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            req = S->tickets[id].req;
        }
        kde_status rc = run_request(S, ctx, st, req);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            Ticket &t = S->tickets[id];
            t.status = rc;
            if (rc != KDE_OK) t.err = kde_last_error(ctx);
            t.t_end = clk::now();
            t.done = true;
            S->in_use -= t.footprint;
            ++S->served;
        }
        S->cv_done.notify_all();
        S->cv_queue.notify_all();
    }
}

extern "C" kde_status kde_server_create(kde_server **out, int device, int32_t n_slots, int64_t hbm_budget_bytes)
{
    if (!out || n_slots < 1 || n_slots > 64 || hbm_budget_bytes <= 0) return KDE_EINVAL;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return KDE_ECUDA;
    kde_server *S = new kde_server();
    S->device = device;
    S->budget = hbm_budget_bytes;
    for (int k = 0; k < n_slots; ++k) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            delete S;
            return KDE_ECUDA;
        }
        kde_ctx *c = nullptr;
        if (kde_create(&c, device, st) != KDE_OK) {
            cudaStreamDestroy(st);
            delete S;
            return KDE_ECUDA;
        }
        S->streams.push_back(st);
        S->ctxs.push_back(c);
    }
    for (int k = 0; k < n_slots; ++k) S->workers.emplace_back(worker_main, S, k);
    *out = S;
    return KDE_OK;
}

extern "C" kde_status kde_server_submit(kde_server *S, const kde_request *req, int64_t *ticket)
{
    if (!S || !req || !ticket) return KDE_EINVAL;
    const kde_request &r = *req;
    bool ok = r.N >= 0 && r.Ng >= 1 && r.Ng <= KDE_MAX_NG && r.L > 0 && (r.N == 0 || r.u);
    switch (r.kind) {
    case KDE_REQ_DEPOSIT: ok = ok && r.out; break;
    case KDE_REQ_GATHER: ok = ok && r.out && r.field; break;
    case KDE_REQ_CV: ok = ok && r.N >= 2 && r.cand && r.n_cand >= 1 && r.n_cand <= 256 && r.out64; break;
    case KDE_REQ_PIC: ok = ok && r.N >= 1 && r.v && r.n_steps >= 0 && r.dt > 0 && r.out64; break;
    default: ok = false;
    }
    if (!ok) return KDE_EINVAL;
    const int64_t fp = request_footprint(r);
    if (fp > S->budget) return KDE_EINVAL;  // could never be admitted
    {
        std::lock_guard<std::mutex> lk(S->mu);
        int64_t id = S->next_id++;
        Ticket &t = S->tickets[id];
        t.req = r;
        t.footprint = fp;
        t.t_submit = clk::now();
        S->queue.push_back(id);
        *ticket = id;
    }
    S->cv_queue.notify_all();
    return KDE_OK;
}

extern "C" kde_status kde_server_wait(kde_server *S, int64_t ticket, double *latency_ms, double *service_ms)
{
    if (!S) return KDE_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return KDE_EINVAL;
    // element references stay valid while other tickets are inserted (iterators may not)
    Ticket &t = it->second;
    S->cv_done.wait(lk, [&] { return t.done; });
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(t.t_end - t.t_submit).count();
    if (service_ms) *service_ms = std::chrono::duration<double, std::milli>(t.t_end - t.t_start).count();
    kde_status rc = t.status;
    S->tickets.erase(ticket);
    return rc;
}

extern "C" kde_status kde_server_destroy(kde_server *S)
{
    if (!S) return KDE_EINVAL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_queue.notify_all();
    for (auto &w : S->workers) w.join();
    for (auto *c : S->ctxs) kde_destroy(c);
    for (auto st : S->streams) cudaStreamDestroy(st);
    delete S;
    return KDE_OK;
}
