// pic.cu -- the electrostatic PIC cycle of Sec. III.A on the device.
//
// Per step (stream-ordered; no host synchronisation except in the AD schedule):
//   [width update: CV over the uniform candidates, kappa* = argmin on the
//    device, leave-one-out pilot densities, Silverman widths + norms]
//   [or the Sec. II.D schedule on the uniform width: Anderson-Darling p-value
//    read on the host, the update rule, CV on optimisation steps, smoothing
//    of h = kappa^{-1/2}]
//   counting sort by cell (positions, velocities, widths, norms, labels)
//   deposit -> int64 grid accumulators
//   Poisson solve straight from the accumulators (mean removed in FP64)
//   gather + leap-frog push + write-back + field energy (one kernel)
#include "common.cuh"

template <typename T>
__global__ void norm_from_kappa_kernel(const T *kappa, int64_t N, T *norm, unsigned int *status, const float2 *ntab)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double k = (double)kappa[i];
    if (!(k > 0 && k <= KDE_KAPPA_MAX)) {
        kde_flag(status, KDE_DEV_KAPPA_RANGE, (unsigned)i);
        k = KDE_KAPPA_MAX;
    }
    // FP32 state: the tabulated norm; FP64 state: the FP64 Bessel series
    if constexpr (sizeof(T) == 4) norm[i] = (T)kde_norm_tab(ntab, (float)k);
    else norm[i] = (T)kde_norm(k);
}

// ---------------------------------------------------------------------------
// Truncation tuner of the FP32 step (no counterpart in the paper: a speed facility).
// Candidate cuts 2^-24 (the reference), 2^-20 and 2^-18 of each kernel's peak; over all
// widths the kernel mass outside them is at most 3.6e-8, 5.8e-7 and 2.3e-6 of the total
// (von Mises tail integrals, worst near kappa = 6-9), below a quarter of the 1e-5
// relative-L2 tolerance of density and field.  On a key's first step every candidate
// runs the deposit + field and a gather (of the reference field) on the step's sorted
// particles, three rounds over the candidates timed by events (the fastest of the last
// two counts).  A candidate is admitted when it changes the results (its window is
// narrower somewhere) and its node field and particle fields match the reference's
// within 2.5e-6 relative L2; it is chosen when it is at least 3% faster than the best
// admitted so far.
// ---------------------------------------------------------------------------
#define CUT_NCAND 3
#define CUT_ERR_TOL 2.5e-6
static const float kCutCand[CUT_NCAND] = {24.f, 20.f, 18.f};

// acc[0] += sum (a - b)^2, acc[1] += sum b^2 (FP64)
__global__ void __launch_bounds__(256) tune_err_kernel(const float *a, const float *b, int64_t n, double *acc)
{
    __shared__ double red[2][8];
    double d2 = 0.0, b2 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = (double)a[i] - (double)b[i];
        d2 += d * d;
        b2 += (double)b[i] * (double)b[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        b2 += __shfl_xor_sync(0xffffffffu, b2, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = d2;
        red[1][warp] = b2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int w = 0; w < 8; ++w) {
            x += red[0][w];
            y += red[1][w];
        }
        atomicAdd(&acc[0], x);
        atomicAdd(&acc[1], y);
    }
}

static kde_status tune_err(kde_ctx *ctx, const float *a, const float *b, int64_t n, double *acc)
{
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = 4LL * (ctx->sm_count > 0 ? ctx->sm_count : 1);
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    tune_err_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(a, b, n, acc);
    KDE_LAUNCHED(ctx, "tune_err_kernel");
    return KDE_OK;
}

static kde_status tune_cut(kde_ctx *ctx, const uint32_t *us, const float *ks, float kappa_u, const float *ns,
                           float norm_u, int64_t N, int Ng, double L, double coef, float w_u, double bound,
                           double charge, bool fd, float &cut)
{
    const size_t ngp = ((size_t)Ng + 63) / 64 * 64, npd = ((size_t)N + 63) / 64 * 64;
    unsigned char *w = (unsigned char *)kde_ws(ctx, WS_TUNE, (2 * ngp + 2 * npd) * 4 + 4 * CUT_NCAND * 8);
    if (!w) return KDE_ENOMEM;
    float *Eref = (float *)w, *Ec = Eref + ngp, *gref = Ec + ngp, *gc = gref + npd;
    double *err = (double *)(gc + npd);
    KDE_CUDA(ctx, cudaMemsetAsync(err, 0, 4 * CUT_NCAND * 8, ctx->stream), "tuner memset");
    constexpr int REPS = 3;  // rounds over the candidates; the first (warm-up) is not timed
    cudaEvent_t ev[REPS][CUT_NCAND + 1];
    for (auto &p : ev)
        for (auto &e : p) KDE_CUDA(ctx, cudaEventCreate(&e), "tuner event");
    kde_status st = KDE_OK;
    // one candidate: deposit + field into E, and a gather of the reference field into g
    auto run = [&](int c, float *E, float *g) -> kde_status {
        DepRows dr{};
        KDE_TRY(kde_deposit_rows_f32(ctx, us, ks, kappa_u, ns, norm_u, N, Ng, coef, w_u, bound, &dr, kCutCand[c]));
        KDE_TRY(kde_field_from_rows(ctx, dr.rows, dr.hdr, dr.G, Ng, L, 1.0 / kde_acc_scale(bound), charge, fd, E));
        return kde_gather_sorted<float>(ctx, us, ks, kappa_u, ns, norm_u, N, Eref, Ng, KDE_TWO_PI / Ng, g, nullptr,
                                        nullptr, kCutCand[c]);
    };
    // the reference first (its field feeds every candidate's gather), then rounds in which
    // the candidates run back to back, so that clock ramps and cache states hit them alike
    st = run(0, Eref, gref);
    for (int rep = 0; rep < REPS && st == KDE_OK; ++rep) {
        for (int c = 0; c < CUT_NCAND && st == KDE_OK; ++c) {
            cudaEventRecord(ev[rep][c], ctx->stream);
            st = run(c, c == 0 ? Eref : Ec, c == 0 ? gref : gc);
            if (st == KDE_OK && rep == 0 && c > 0) st = tune_err(ctx, Ec, Eref, Ng, err + 4 * c);
            if (st == KDE_OK && rep == 0 && c > 0) st = tune_err(ctx, gc, gref, N, err + 4 * c + 2);
        }
        cudaEventRecord(ev[rep][CUT_NCAND], ctx->stream);
    }
    double eh[4 * CUT_NCAND];
    if (st == KDE_OK) {
        cudaError_t e = cudaMemcpyAsync(eh, err, sizeof(eh), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = kde_cuda_check(ctx, e, "tuner results");
    }
    if (st == KDE_OK) {
        float t[CUT_NCAND];
        for (int c = 0; c < CUT_NCAND; ++c) {
            t[c] = 3.0e38f;
            for (int rep = 1; rep < REPS; ++rep) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[rep][c], ev[rep][c + 1]);
                t[c] = ms < t[c] ? ms : t[c];
            }
        }
        // a candidate must change the computation (a narrower window somewhere), stay
        // within the error bound, and beat the best admitted time by 3%
        auto rel = [](double d2, double b2) { return d2 == 0.0 ? 0.0 : (b2 > 0.0 ? sqrt(d2 / b2) : 1.0e300); };
        int best = 0;
        for (int c = 1; c < CUT_NCAND; ++c) {
            const bool changed = eh[4 * c] > 0.0 || eh[4 * c + 2] > 0.0;
            const bool ok = rel(eh[4 * c], eh[4 * c + 1]) <= CUT_ERR_TOL && rel(eh[4 * c + 2], eh[4 * c + 3]) <= CUT_ERR_TOL;
            if (changed && ok && t[c] < 0.97f * t[best]) best = c;
        }
        cut = kCutCand[best];
    }
    for (auto &p : ev)
        for (auto &e : p) cudaEventDestroy(e);
    return st;
}

// standard PIC with a B-spline shape: deposit, Poisson, energy, gather + push
static kde_status pic_run_bspline(kde_ctx *ctx, pic_state *st, int n_steps)
{
    const int64_t N = st->N;
    const int Ng = st->Ng;
    const double L = st->L;
    const double h = st->shape_h > 0 ? st->shape_h : L / Ng;
    const bool fd = (st->flags & KDE_POISSON_FD) != 0;
    long long *acc = (long long *)kde_ws(ctx, WS_ACC, (size_t)Ng * 8);
    float *E = (float *)kde_ws(ctx, WS_GRID0, (size_t)Ng * sizeof(float));
    if (!acc || !E) return KDE_ENOMEM;
    for (int s = 0; s < n_steps; ++s) {
        const int64_t step = st->step;
        double bound = 0.0;
        KDE_TRY(kde_bspline_deposit_acc(ctx, st->u, N, st->shape_order, h, Ng, L, acc, &bound));
        KDE_TRY(kde_poisson_impl<float>(ctx, nullptr, acc, 1.0 / kde_acc_scale(bound), Ng, L, st->charge,
                                        st->background, fd, E));
        if (st->energy) KDE_TRY(kde_energy_impl<float>(ctx, E, Ng, L, st->energy + step));
        const double kick = (step == 0 && !(st->flags & PIC_NO_BACKSTEP)) ? 0.5 : 1.0;
        KDE_TRY(kde_bspline_gather_push(ctx, st->u, (float *)st->v, N, st->shape_order, h, Ng, L, E,
                                        kick * st->qm * st->dt, st->dt * 4294967296.0 / L));
        st->step = step + 1;
    }
    return KDE_OK;
}

template <typename T>
static kde_status pic_run(kde_ctx *ctx, pic_state *st, int n_steps)
{
    const int64_t N = st->N;
    const int Ng = st->Ng;
    const double L = st->L;
    const bool per = st->kappa != nullptr;
    const bool adsched = st->width_ad != 0;
    const bool sched = !adsched && st->width_every > 0 && st->n_cand > 0;
    const bool fd = (st->flags & KDE_POISSON_FD) != 0;
    T *norm_arr = (T *)st->kappa_norm;
    // CV form of the schedule: forced by a flag, else the cheaper exact form (cost rule)
    const bool cv_spec = (st->flags & KDE_CV_SPECTRAL) ||
                         (!(st->flags & KDE_CV_PAIRS) && st->n_cand > 0 && st->cand &&
                          kde_cv_prefer_spectral(N, st->cand, st->n_cand));

    // the width update (CV) shares the sort slots; size them for it up front and
    // fetch the pointers again after every update, since a slot may be regrown
    const size_t npad = (size_t)((N + 255) / 256) * 256;
    // two sets of sorted widths, norms and labels, used in turn: within a call the push
    // writes them back to the state only on the call's last step, and each step sorts
    // them from wherever the previous step left them
    uint32_t *us = nullptr, *ids2[2] = {nullptr, nullptr};
    T *vs = nullptr, *ks2[2] = {nullptr, nullptr}, *ns2[2] = {nullptr, nullptr};
    auto fetch_ws = [&]() -> bool {
        us = (uint32_t *)kde_ws(ctx, WS_SORT_U, npad * 4);
        vs = (T *)kde_ws(ctx, WS_SORT_P0, npad * sizeof(T));
        bool ok = us && vs;
        for (int b = 0; b < 2; ++b) {
            ks2[b] = per ? (T *)kde_ws(ctx, b ? WS_SORT_P1B : WS_SORT_P1, npad * sizeof(T)) : nullptr;
            ns2[b] = per ? (T *)kde_ws(ctx, b ? WS_SORT_P2B : WS_SORT_P2, npad * sizeof(T)) : nullptr;
            ids2[b] = st->id ? (uint32_t *)kde_ws(ctx, b ? WS_SORT_P3B : WS_SORT_P3, npad * 4) : nullptr;
            ok = ok && (!per || (ks2[b] && ns2[b])) && (!st->id || ids2[b]);
        }
        return ok;
    };
    if (!fetch_ws()) return KDE_ENOMEM;
    long long *acc = (long long *)kde_ws(ctx, WS_ACC, (size_t)Ng * 8);
    T *E = (T *)kde_ws(ctx, WS_GRID0, (size_t)Ng * sizeof(T));
    float *loo = sched ? (float *)kde_ws(ctx, WS_PIC_LOO, (size_t)N * 4) : nullptr;
    double *ks_dev = sched ? (double *)kde_ws(ctx, WS_PIC_KS, 64) : nullptr;
    double *cv_dev = (sched || adsched) ? (double *)kde_ws(ctx, WS_CV_OUT, (size_t)st->n_cand * 8 + 64) : nullptr;
    double *ad_out = adsched ? (double *)kde_ws(ctx, WS_AD_OUT, 16) : nullptr;
    if (!acc || !E || (sched && (!loo || !ks_dev || !cv_dev)) || (adsched && (!cv_dev || !ad_out)))
        return KDE_ENOMEM;
    int *amin_dev = (sched || adsched) ? (int *)(cv_dev + st->n_cand) : nullptr;
    // the AD schedule smooths h = kappa^{-1/2}, carried across the steps of this call
    double h_ad = adsched ? 1.0 / sqrt(st->kappa_uniform) : 0.0;

    if (per) {
        norm_from_kappa_kernel<T><<<(unsigned)((N + 255) / 256), 256, 0, ctx->stream>>>(
            (const T *)st->kappa, N, norm_arr, ctx->d_status, ctx->norm_tab);
        KDE_LAUNCHED(ctx, "norm_from_kappa_kernel");
    }
    const double coef = KDE_TWO_PI / L;
    const double w_u = L / (double)N;
    // the FP32 gather + push adds the next step's sort counts; a step whose table was
    // overwritten since (first step of the call, CV or AD sorts) counts afresh
    bool counted = false;
    // where the current widths, norms and labels are: the state's arrays, or one of the
    // two sorted sets
    const T *k_cur = per ? (const T *)st->kappa : nullptr;
    const T *n_cur = per ? (const T *)norm_arr : nullptr;
    const uint32_t *id_cur = st->id;
    for (int s = 0; s < n_steps; ++s) {
        const int64_t step = st->step;
        const bool update = sched && step % st->width_every == 0;
        if (update) {
            counted = false;  // the CV's own sort reuses the count table
            KdeRange r_("kdepic width update (CV + Silverman)");
            if (cv_spec)
                KDE_TRY(kde_cv_spectral_device(ctx, st->u, N, L, st->cand, st->n_cand, cv_dev, amin_dev, loo, ks_dev));
            else
                KDE_TRY(kde_cv_device(ctx, st->u, nullptr, N, L, st->cand, st->n_cand, false, cv_dev, amin_dev, loo,
                                      ks_dev));
            KDE_TRY(kde_adapt_device(ctx, loo, N, L, ks_dev, 0.0, st->alpha, st->kappa_min, st->kappa_max, st->kappa,
                                     norm_arr, sizeof(T) == 8));
            k_cur = (const T *)st->kappa;  // the new widths and norms are in the state's arrays
            n_cur = (const T *)norm_arr;
            if (!fetch_ws()) return KDE_ENOMEM;
        }
        if (adsched) {
            counted = false;  // the AD test's radix sort reuses the count table
            KdeRange r_("kdepic Anderson-Darling schedule");
            KDE_TRY(kde_ad_device(ctx, st->u, N, ad_out, st->ad_log_p ? st->ad_log_p + step : nullptr));
            double ad_h[2];
            KDE_CUDA(ctx, cudaMemcpyAsync(ad_h, ad_out, 16, cudaMemcpyDeviceToHost, ctx->stream), "AD result copy");
            KDE_TRY(kde_sync(ctx));
            const double lp = ad_h[1], l2t = log(2.0 * st->ad_threshold);
            if (st->ad_log_pth >= 0.0) st->ad_log_pth = l2t;
            bool opt = false;
            if (lp > l2t) {
                st->ad_log_pth = l2t;
            } else if (lp < st->ad_log_pth - log(2.0)) {
                st->ad_log_pth = lp;
                opt = true;
            }
            if (opt) {
                if (cv_spec)
                    KDE_TRY(kde_cv_spectral_device(ctx, st->u, N, L, st->cand, st->n_cand, cv_dev, amin_dev, nullptr,
                                                   nullptr));
                else
                    KDE_TRY(kde_cv_device(ctx, st->u, nullptr, N, L, st->cand, st->n_cand, false, cv_dev, amin_dev,
                                          nullptr, nullptr));
                int am = 0;
                KDE_CUDA(ctx, cudaMemcpyAsync(&am, amin_dev, 4, cudaMemcpyDeviceToHost, ctx->stream), "argmin copy");
                KDE_TRY(kde_sync(ctx));
                const double ht = 1.0 / sqrt(st->cand[am]);
                if (!(st->h_target > 0.0)) h_ad = ht;
                st->h_target = ht;
                ++st->n_opt;
                if (!fetch_ws()) return KDE_ENOMEM;
            }
            if (st->h_target > 0.0) h_ad = st->adjust_rate * st->h_target + (1.0 - st->adjust_rate) * h_ad;
            st->kappa_uniform = 1.0 / (h_ad * h_ad);
        }
        // this step's sorted set: the one the current arrays are not in
        auto holds = [&](int b) {
            return (per && (k_cur == ks2[b] || n_cur == ns2[b])) || (st->id && id_cur == ids2[b]);
        };
        const int wsel = holds(0) ? 1 : 0;
        T *ks = ks2[wsel], *ns = ns2[wsel];
        uint32_t *ids = ids2[wsel];
        const bool last = s == n_steps - 1;
        SortPayload pl[4];
        int npl = 0;
        pl[npl++] = SortPayload{st->v, vs, (int)sizeof(T)};
        if (per) {
            pl[npl++] = SortPayload{k_cur, ks, (int)sizeof(T)};
            pl[npl++] = SortPayload{n_cur, ns, (int)sizeof(T)};
        }
        if (st->id) pl[npl++] = SortPayload{id_cur, ids, 4};
        {
            KdeRange r_("kdepic sort by cell");
            KDE_TRY(kde_sort_by_bin(ctx, st->u, N, Ng, us, pl, npl, nullptr, counted));
        }

        const double norm_u = per ? 0.0 : kde_norm(st->kappa_uniform);
        const double norm_bound = per ? kde_norm(KDE_KAPPA_MAX) : norm_u;
        const double bound = (double)N * w_u * coef * norm_bound;
        float cut = 0.f;  // FP32 truncation cut exponent of this step's deposit and gather
        if constexpr (sizeof(T) == 4) {
            cut = kde_fp32_cut(ctx);
            if (!(ctx->cut_fixed > 0.0)) {
                const uint64_t key = kde_width_key(N, Ng, per, st->kappa_uniform);
                auto it = ctx->cut_tuned.find(key);
                if (it != ctx->cut_tuned.end()) {
                    cut = it->second;
                } else if (ctx->autotune) {
                    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
                    cudaStreamIsCapturing(ctx->stream, &cap);
                    if (cap == cudaStreamCaptureStatusNone) {
                        KdeRange r_("kdepic truncation tuner");
                        KDE_TRY(tune_cut(ctx, us, (const float *)ks, (float)st->kappa_uniform, (const float *)ns,
                                         (float)norm_u, N, Ng, L, coef, (float)w_u, bound, st->charge, fd,
                                         cut));
                        ctx->cut_tuned[key] = cut;
                    }
                }
            }
            // FP32: per-CTA rows, summed inside the field kernel (no accumulator round trip)
            DepRows dr{};
            {
                KdeRange r_("kdepic deposit");
                KDE_TRY(kde_deposit_rows_f32(ctx, us, ks, (float)st->kappa_uniform, ns, (float)norm_u, N, Ng, coef,
                                             (float)w_u, bound, &dr, cut));
            }
            {
                KdeRange r_("kdepic field (row sums + Poisson)");
                KDE_TRY(kde_field_from_rows(ctx, dr.rows, dr.hdr, dr.G, Ng, L, 1.0 / kde_acc_scale(bound), st->charge,
                                            fd, (float *)E));
            }
        } else {
            {
                KdeRange r_("kdepic deposit");
                KDE_TRY(kde_deposit_sorted<T>(ctx, us, ks, (T)st->kappa_uniform, ns, (T)norm_u, nullptr, (T)w_u, N,
                                              Ng, coef, acc, bound, nullptr, norm_bound));
            }
            {
                KdeRange r_("kdepic Poisson");
                KDE_TRY(kde_poisson_impl<T>(ctx, nullptr, acc, 1.0 / kde_acc_scale(bound), Ng, L, st->charge,
                                            st->background, fd, E));
            }
        }

        PushArgs pa{};
        pa.v_in = vs;
        pa.u_out = st->u;
        pa.v_out = st->v;
        // widths, norms and labels go back to the state only on the call's last step
        pa.kappa_out = (per && last) ? st->kappa : nullptr;
        pa.norm_in = ns;
        pa.norm_out = (per && last) ? norm_arr : nullptr;
        pa.id_in = ids;
        pa.id_out = last ? st->id : nullptr;
        pa.kick = (step == 0 && !(st->flags & PIC_NO_BACKSTEP)) ? 0.5 : 1.0;
        pa.qm_dt = st->qm * st->dt;
        pa.dt_scale = st->dt * 4294967296.0 / L;
        pa.energy = st->energy ? st->energy + step : nullptr;
        // the CV width in force: this step's update, else the previous step's history entry
        // (the state's own record; the context's copy may belong to another state), else the
        // context's copy (no history kept, so the value is not reported anywhere)
        pa.kstar_in = update ? ks_dev
                             : (sched && st->kappa_star && step > 0 ? st->kappa_star + step - 1 : (sched ? ks_dev : nullptr));
        pa.kstar_out = st->kappa_star ? st->kappa_star + step : nullptr;
        pa.dx = L / Ng;
        pa.xcut = cut;
        SortCounts sc{};
        if constexpr (sizeof(T) == 4) {
            KDE_TRY(kde_sort_counts_table(ctx, N, Ng, &sc));
            pa.counts = sc.counts;
            pa.cnt_nblk = sc.nblk;
            pa.cnt_shift = sc.tile_shift;
        }
        {
            KdeRange r_("kdepic gather + push");
            KDE_TRY(kde_gather_sorted<T>(ctx, us, ks, (T)st->kappa_uniform, ns, (T)norm_u, N, E, Ng,
                                         KDE_TWO_PI / Ng, nullptr, nullptr, &pa));
        }
        counted = pa.counts != nullptr;
        if (!last) {  // the sorted set now holds the current widths, norms and labels
            k_cur = ks;
            n_cur = ns;
            id_cur = ids;
        }
        st->step = step + 1;
    }
    return KDE_OK;
}

extern "C" kde_status pic_step(kde_ctx *ctx, pic_state *st, int32_t n_steps)
{
    if (!ctx) return KDE_EINVAL;
    if (!st || n_steps < 0) return kde_fail(ctx, KDE_EINVAL, "pic_step: null state or negative step count");
    if (st->N < 1 || st->N > 0xFFFFFFFFll || st->Ng < 1 || st->Ng > KDE_MAX_NG || !(st->L > 0) || !(st->dt > 0) ||
        !st->u || !st->v || st->step < 0)
        return kde_fail(ctx, KDE_EINVAL, "pic_step: need 1 <= N < 2^32, 1 <= Ng <= %d, L > 0, dt > 0, u and v",
                        KDE_MAX_NG);
    if (st->flags & ~(KDE_F64 | KDE_POISSON_FD | KDE_CV_SPECTRAL | KDE_CV_PAIRS | PIC_NO_BACKSTEP))
        return kde_fail(ctx, KDE_ENOTSUP, "pic_step: unsupported flags 0x%x", st->flags);
    if ((st->flags & KDE_CV_SPECTRAL) && (st->flags & KDE_CV_PAIRS))
        return kde_fail(ctx, KDE_EINVAL, "pic_step: KDE_CV_SPECTRAL and KDE_CV_PAIRS exclude each other");
    if (st->width_ad) {
        if (st->kappa || !st->cand || st->n_cand < 1 || st->n_cand > 256 || st->N < KDE_AD_MIN_N ||
            !(st->ad_threshold > 0 && st->ad_threshold < 0.5) || !(st->adjust_rate > 0 && st->adjust_rate <= 1))
            return kde_fail(ctx, KDE_EINVAL,
                            "pic_step: the Anderson-Darling schedule needs a uniform width (kappa == NULL), 1..256 "
                            "host candidates, N >= %d, 0 < ad_threshold < 0.5 and 0 < adjust_rate <= 1",
                            KDE_AD_MIN_N);
        for (int c = 0; c < st->n_cand; ++c)
            if (!(st->cand[c] > 0 && st->cand[c] <= KDE_KAPPA_MAX))
                return kde_fail(ctx, KDE_EINVAL, "pic_step: candidate %d outside (0, 1e6]", c);
    }
    if (st->kappa && !st->kappa_norm)
        return kde_fail(ctx, KDE_EINVAL, "pic_step: per-particle widths need the kappa_norm array");
    if (!st->kappa && st->shape_order == 0 && !(st->kappa_uniform > 0 && st->kappa_uniform <= KDE_KAPPA_MAX))
        return kde_fail(ctx, KDE_EINVAL, "pic_step: kappa_uniform must be in (0, 1e6]");
    if (!st->width_ad && st->width_every > 0 && st->n_cand > 0) {
        if (!st->kappa || !st->cand || st->n_cand > 256 || st->N < 2 || !(st->alpha >= 0) ||
            !(st->kappa_min <= st->kappa_max))
            return kde_fail(ctx, KDE_EINVAL,
                            "pic_step: the width schedule needs a kappa array, 1..256 host candidates, N >= 2, "
                            "alpha >= 0 and kappa_min <= kappa_max");
        for (int c = 0; c < st->n_cand; ++c)
            if (!(st->cand[c] > 0 && st->cand[c] <= KDE_KAPPA_MAX))
                return kde_fail(ctx, KDE_EINVAL, "pic_step: candidate %d outside (0, 1e6]", c);
    }
    if (st->shape_order != 0) {
        const double h = st->shape_h > 0 ? st->shape_h : st->L / st->Ng;
        if (!(st->shape_order == 1 || st->shape_order == 2 || st->shape_order == 3 || st->shape_order == 5) ||
            !((st->shape_order + 1) * h < st->L) || st->shape_h < 0 || (st->flags & KDE_F64) || st->kappa ||
            st->width_ad || (st->width_every > 0 && st->n_cand > 0))
            return kde_fail(ctx, KDE_EINVAL,
                            "pic_step: a B-spline shape needs order in {1, 2, 3, 5}, 0 < (order+1) h < L, FP32, "
                            "no particle-wise widths and no width schedule");
        cudaSetDevice(ctx->device);
        return pic_run_bspline(ctx, st, n_steps);
    }
    cudaSetDevice(ctx->device);
    if (st->flags & KDE_F64) return pic_run<double>(ctx, st, n_steps);
    return pic_run<float>(ctx, st, n_steps);
}

// ---------------------------------------------------------------------------
// pic_step on a host-resident state: copy in, run on the device, copy out
// ---------------------------------------------------------------------------
extern "C" kde_status pic_step_host(kde_ctx *ctx, pic_state *st, int32_t n_steps)
{
    if (!ctx) return KDE_EINVAL;
    if (!st || n_steps < 0 || st->N < 1 || st->N > 0xFFFFFFFFll || !st->u || !st->v || st->step < 0)
        return kde_fail(ctx, KDE_EINVAL, "pic_step_host: need a state with 1 <= N < 2^32, u, v and step >= 0");
    cudaSetDevice(ctx->device);
    const size_t N = (size_t)st->N;
    const size_t el = (st->flags & KDE_F64) ? 8 : 4;
    const size_t hist = (size_t)st->step + (size_t)n_steps;  // histories are indexed by step
    pic_state d = *st;
    d.u = (uint32_t *)kde_ws(ctx, WS_HOST_U, N * 4);
    d.v = kde_ws(ctx, WS_HOST_V, N * el);
    d.kappa = st->kappa ? kde_ws(ctx, WS_HOST_K, N * el) : nullptr;
    d.kappa_norm = st->kappa ? kde_ws(ctx, WS_HOST_NORM, N * el) : nullptr;
    d.id = st->id ? (uint32_t *)kde_ws(ctx, WS_HOST_ID, N * 4) : nullptr;
    const int nh = (st->energy ? 1 : 0) + (st->kappa_star ? 1 : 0) + (st->ad_log_p ? 1 : 0);
    double *h = nh ? (double *)kde_ws(ctx, WS_HOST_HIST, (size_t)nh * (hist > 0 ? hist : 1) * 8) : nullptr;
    if (!d.u || !d.v || (st->kappa && (!d.kappa || !d.kappa_norm)) || (st->id && !d.id) || (nh && !h))
        return KDE_ENOMEM;
    int k = 0;
    d.energy = st->energy ? h + (k++) * hist : nullptr;
    d.kappa_star = st->kappa_star ? h + (k++) * hist : nullptr;
    d.ad_log_p = st->ad_log_p ? h + (k++) * hist : nullptr;
    cudaStream_t s = ctx->stream;
    KDE_CUDA(ctx, cudaMemcpyAsync(d.u, st->u, N * 4, cudaMemcpyHostToDevice, s), "state copy in");
    KDE_CUDA(ctx, cudaMemcpyAsync(d.v, st->v, N * el, cudaMemcpyHostToDevice, s), "state copy in");
    if (st->kappa) KDE_CUDA(ctx, cudaMemcpyAsync(d.kappa, st->kappa, N * el, cudaMemcpyHostToDevice, s), "state copy in");
    if (st->id) KDE_CUDA(ctx, cudaMemcpyAsync(d.id, st->id, N * 4, cudaMemcpyHostToDevice, s), "state copy in");
    // the width in force before this call is the previous step's history entry
    if (st->kappa_star && st->step > 0)
        KDE_CUDA(ctx, cudaMemcpyAsync(d.kappa_star + st->step - 1, st->kappa_star + st->step - 1, 8,
                                      cudaMemcpyHostToDevice, s), "history copy in");
    KDE_TRY(pic_step(ctx, &d, n_steps));
    KDE_CUDA(ctx, cudaMemcpyAsync(st->u, d.u, N * 4, cudaMemcpyDeviceToHost, s), "state copy out");
    KDE_CUDA(ctx, cudaMemcpyAsync(st->v, d.v, N * el, cudaMemcpyDeviceToHost, s), "state copy out");
    if (st->kappa) KDE_CUDA(ctx, cudaMemcpyAsync(st->kappa, d.kappa, N * el, cudaMemcpyDeviceToHost, s), "state copy out");
    if (st->id) KDE_CUDA(ctx, cudaMemcpyAsync(st->id, d.id, N * 4, cudaMemcpyDeviceToHost, s), "state copy out");
    const size_t off = (size_t)st->step, cnt = (size_t)n_steps * 8;
    if (n_steps > 0) {
        if (st->energy)
            KDE_CUDA(ctx, cudaMemcpyAsync(st->energy + off, d.energy + off, cnt, cudaMemcpyDeviceToHost, s), "copy out");
        if (st->kappa_star)
            KDE_CUDA(ctx, cudaMemcpyAsync(st->kappa_star + off, d.kappa_star + off, cnt, cudaMemcpyDeviceToHost, s),
                     "copy out");
        if (st->ad_log_p)
            KDE_CUDA(ctx, cudaMemcpyAsync(st->ad_log_p + off, d.ad_log_p + off, cnt, cudaMemcpyDeviceToHost, s),
                     "copy out");
    }
    const kde_status rc = kde_sync(ctx);
    // the scalar state the run advanced
    st->step = d.step;
    st->kappa_uniform = d.kappa_uniform;
    st->ad_log_pth = d.ad_log_pth;
    st->h_target = d.h_target;
    st->n_opt = d.n_opt;
    return rc;
}
