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
//
// HBM accounting.  Device memory committed at any time is the transient
// buffers of the running requests plus the workspace every slot's context
// holds (a context keeps its workspace between requests).  A request's
// footprint is split into its transient buffers and the workspace it needs; a
// slot admits the head request when the committed total plus the buffers plus
// the slot's workspace growth fits the budget.  When only the workspace held by
// idle slots stands in the way, those slots' workspaces are released first.
// After each request the slot's actual workspace is measured again, so growth
// beyond the estimate is charged to later admissions.
#include <chrono>
#include <condition_variable>
#include <cstring>
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
    bool cancelled = false;
    int64_t io = 0;  // transient device buffers
    int64_t ws = 0;  // workspace the request needs in its slot's context
    double dev_start = -1.0, dev_end = -1.0;  // device clock, ms since the server's epoch event
    std::string err;
};

}  // namespace

struct kde_server {
    int device = 0;
    int64_t budget = 0;
    int64_t io_in_use = 0;         // transient buffers of the running requests
    int64_t committed_peak = 0;    // largest committed total seen at an admission
    std::vector<int64_t> held;     // workspace each slot's context holds (or has reserved)
    std::vector<char> busy;
    std::vector<std::thread> workers;
    std::vector<kde_ctx *> ctxs;
    std::vector<cudaStream_t> streams;
    cudaEvent_t epoch = nullptr;   // device-clock origin of the request intervals
    std::mutex mu;
    std::condition_variable cv_queue, cv_done;
    std::deque<int64_t> queue;
    std::unordered_map<int64_t, Ticket> tickets;
    int64_t next_id = 1;
    bool stop = false;
    int64_t served = 0, cancelled = 0, trims = 0;
};

// transient device buffers of a request (inputs and outputs), in bytes
static int64_t request_io_bytes(const kde_request &r)
{
    const int64_t N = r.N, Ng = r.Ng;
    int64_t b = N * 4 + (r.kappa ? N * 4 : 0) + 4096;
    switch (r.kind) {
    case KDE_REQ_DEPOSIT: b += Ng * 4; break;
    case KDE_REQ_GATHER: b += Ng * 4 + N * 4; break;
    case KDE_REQ_PIC: b += N * 4 + (r.kappa ? N * 4 : 0) + (int64_t)(r.n_steps > 0 ? r.n_steps : 1) * 8; break;
    default: break;
    }
    return b;
}

// workspace a request of this size grows in its slot's context (sort copies, CV
// tables, grid scratch), in bytes: an upper estimate of what the kernels request
static int64_t request_ws_bytes(const kde_request &r)
{
    const int64_t N = r.N, Ng = r.Ng;
    // (workspace slots grow by a quarter beyond the request, hence the margins)
    if (r.kind == KDE_REQ_CV)
        return N * (32 + 5 * (int64_t)r.n_cand) + (int64_t)r.n_cand * 8192 * 10 + (4 << 20);
    // sort slots (two sets of widths and norms for PIC runs), and the persistent deposit's
    // int64 rows (an upper bound: 640 rows of Ng entries)
    return N * 56 + Ng * (64 + 640 * 8) + (16 << 20);
}

// device memory a context holds: its workspace slots and cached tables
static int64_t ctx_held_bytes(const kde_ctx *c)
{
    int64_t b = 0;
    for (int i = 0; i < WS_NSLOTS; ++i) b += (int64_t)c->ws_bytes[i];
    for (auto &kv : c->node_tab) b += (int64_t)kv.first.first * (kv.first.second ? 16 : 8);
    for (auto &kv : c->green_tab) b += (int64_t)std::get<0>(kv.first) * (std::get<3>(kv.first) ? 8 : 4);
    return b;
}

// release the workspace of a context whose slot is idle (its stream has drained)
static void ctx_trim(kde_ctx *c)
{
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (int i = 0; i < WS_NSLOTS; ++i)
        if (c->ws[i]) {
            cudaFree(c->ws[i]);
            c->ws[i] = nullptr;
            c->ws_bytes[i] = 0;
        }
    c->sp_atab = nullptr;  // held in a workspace slot
    c->sp_atab_cands.clear();
}

static kde_status run_request(kde_server *S, kde_ctx *ctx, cudaStream_t st, const kde_request &r, cudaEvent_t ev0,
                              cudaEvent_t ev1)
{
    const int64_t N = r.N;
    cudaEventRecord(ev0, st);
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
    cudaEventRecord(ev1, st);
    kde_status s2 = kde_sync(ctx);
    if (rc == KDE_OK) rc = s2;
    (void)S;
    return rc;
}

// admission of the queue's head on idle slot `slot` (called with the lock held)
static bool admit_head(kde_server *S, int slot)
{
    if (S->queue.empty()) return false;
    Ticket &t = S->tickets[S->queue.front()];
    auto committed = [&]() {
        int64_t c = S->io_in_use;
        for (int64_t h : S->held) c += h;
        return c;
    };
    const int64_t grow = t.ws > S->held[slot] ? t.ws - S->held[slot] : 0;
    bool anyone_busy = false;
    for (char b : S->busy) anyone_busy = anyone_busy || b;
    if (committed() + t.io + grow > S->budget) {
        // release the workspace of the other idle slots, then look again
        for (size_t k = 0; k < S->held.size(); ++k)
            if ((int)k != slot && !S->busy[k] && S->held[k] > 0) {
                ctx_trim(S->ctxs[k]);
                S->held[k] = ctx_held_bytes(S->ctxs[k]);
                ++S->trims;
            }
        if (committed() + t.io + grow > S->budget) {
            if (anyone_busy) return false;
            // nothing else runs: start from this slot's own empty workspace too (the
            // request fits the budget by itself: kde_server_submit refuses larger ones)
            ctx_trim(S->ctxs[slot]);
            S->held[slot] = ctx_held_bytes(S->ctxs[slot]);
            ++S->trims;
        }
    }
    const int64_t grow2 = t.ws > S->held[slot] ? t.ws - S->held[slot] : 0;
    S->io_in_use += t.io;
    S->held[slot] += grow2;
    const int64_t c = committed();
    if (c > S->committed_peak) S->committed_peak = c;
    return true;
}

static void worker_main(kde_server *S, int slot)
{
    cudaSetDevice(S->device);
    kde_ctx *ctx = S->ctxs[slot];
    cudaStream_t st = S->streams[slot];
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    for (;;) {
        int64_t id;
        kde_request req;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            // FIFO admission: the head request starts when its footprint fits the budget
            // (admit_head commits the accounting when it returns true); a stopping server
            // still finishes its queue
            bool admitted = false;
            S->cv_queue.wait(lk, [&] {
                admitted = admit_head(S, slot);
                return admitted || (S->stop && S->queue.empty());
            });
            if (!admitted) break;
            id = S->queue.front();
            S->queue.pop_front();
            Ticket &t = S->tickets[id];
            S->busy[slot] = 1;
            t.t_start = clk::now();
            req = t.req;
        }
        kde_status rc = run_request(S, ctx, st, req, ev0, ev1);
        float a = -1.f, b = -1.f;
        if (cudaEventElapsedTime(&a, S->epoch, ev0) != cudaSuccess || cudaEventElapsedTime(&b, S->epoch, ev1) != cudaSuccess) {
            cudaGetLastError();
            a = b = -1.f;
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            Ticket &t = S->tickets[id];
            t.status = rc;
            if (rc != KDE_OK) t.err = kde_last_error(ctx);
            t.t_end = clk::now();
            t.dev_start = a;
            t.dev_end = b;
            t.done = true;
            S->io_in_use -= t.io;
            S->held[slot] = ctx_held_bytes(ctx);
            S->busy[slot] = 0;
            ++S->served;
        }
        S->cv_done.notify_all();
        S->cv_queue.notify_all();
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
}

extern "C" kde_status kde_server_create(kde_server **out, int device, int32_t n_slots, int64_t hbm_budget_bytes)
{
    if (!out || n_slots < 1 || n_slots > 64 || hbm_budget_bytes <= 0) return KDE_EINVAL;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return KDE_ECUDA;
    kde_server *S = new kde_server();
    S->device = device;
    S->budget = hbm_budget_bytes;
    if (cudaEventCreate(&S->epoch) != cudaSuccess) {
        delete S;
        return KDE_ECUDA;
    }
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
        S->held.push_back(ctx_held_bytes(c));
        S->busy.push_back(0);
    }
    cudaEventRecord(S->epoch, S->streams[0]);
    cudaEventSynchronize(S->epoch);
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
    const int64_t io = request_io_bytes(r), ws = request_ws_bytes(r);
    if (io + ws + (1 << 20) > S->budget) return KDE_EINVAL;  // could never be admitted (1 MiB for tables)
    {
        std::lock_guard<std::mutex> lk(S->mu);
        int64_t id = S->next_id++;
        Ticket &t = S->tickets[id];
        t.req = r;
        t.io = io;
        t.ws = ws;
        t.t_submit = clk::now();
        S->queue.push_back(id);
        *ticket = id;
    }
    S->cv_queue.notify_all();
    return KDE_OK;
}

extern "C" kde_status kde_server_wait_msg(kde_server *S, int64_t ticket, double *times, char *msg, int32_t msg_cap)
{
    if (!S || msg_cap < 0 || (msg_cap > 0 && !msg)) return KDE_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return KDE_EINVAL;
    // element references stay valid while other tickets are inserted (iterators may not)
    Ticket &t = it->second;
    S->cv_done.wait(lk, [&] { return t.done; });
    if (times) {
        times[0] = std::chrono::duration<double, std::milli>(t.t_end - t.t_submit).count();
        times[1] = t.cancelled ? 0.0 : std::chrono::duration<double, std::milli>(t.t_end - t.t_start).count();
        times[2] = t.dev_start;
        times[3] = t.dev_end;
    }
    kde_status rc = t.status;
    if (msg_cap > 0) {
        const std::string m = rc == KDE_OK ? std::string() : (t.err.empty() ? std::string("request failed") : t.err);
        const size_t n = m.size() < (size_t)msg_cap - 1 ? m.size() : (size_t)msg_cap - 1;
        memcpy(msg, m.data(), n);
        msg[n] = 0;
    }
    S->tickets.erase(ticket);
    return rc;
}

extern "C" kde_status kde_server_wait_times(kde_server *S, int64_t ticket, double *times)
{
    return kde_server_wait_msg(S, ticket, times, nullptr, 0);
}

extern "C" kde_status kde_server_wait(kde_server *S, int64_t ticket, double *latency_ms, double *service_ms)
{
    double t[4] = {0, 0, -1, -1};
    kde_status rc = kde_server_wait_times(S, ticket, t);
    if (latency_ms) *latency_ms = t[0];
    if (service_ms) *service_ms = t[1];
    return rc;
}

extern "C" kde_status kde_server_cancel(kde_server *S, int64_t ticket)
{
    if (!S) return KDE_EINVAL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->tickets.find(ticket);
        if (it == S->tickets.end()) return KDE_EINVAL;
        auto q = std::find(S->queue.begin(), S->queue.end(), ticket);
        if (q == S->queue.end()) return KDE_EBUSY;  // admitted already (running or done)
        S->queue.erase(q);
        Ticket &t = it->second;
        t.cancelled = true;
        t.status = KDE_ECANCELED;
        t.t_start = t.t_end = clk::now();
        t.done = true;
        ++S->cancelled;
    }
    S->cv_done.notify_all();
    S->cv_queue.notify_all();  // the next request may now be the head
    return KDE_OK;
}

extern "C" kde_status kde_server_stats(kde_server *S, int64_t *stats)
{
    if (!S || !stats) return KDE_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    int64_t held = 0;
    for (int64_t h : S->held) held += h;
    stats[0] = S->io_in_use + held;
    stats[1] = S->committed_peak;
    stats[2] = S->budget;
    stats[3] = S->served;
    stats[4] = S->cancelled;
    stats[5] = (int64_t)S->queue.size();
    stats[6] = S->trims;
    stats[7] = held;
    return KDE_OK;
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
    if (S->epoch) cudaEventDestroy(S->epoch);
    delete S;
    return KDE_OK;
}
