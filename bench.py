#!/usr/bin/env python
"""Benchmark of the KDE-PIC hot path on one GB300 (or N independent replicas).

Default line (`--workload landau`): the Landau-damping run with particle-wise widths --
N = 2^20 electrons, Ng = 256 nodes, L = 4 pi (k = 0.5), density 1 + 0.05 cos(kx),
Maxwellian v_th = 1, dt = 0.1, 1000 steps; every 50 steps the width is re-selected by
leave-one-out CV over 64 candidates log-spaced in [1, 1e4] and Silverman's particle-wise
widths (alpha = 0.5) are recomputed.  One benchmark step is the whole 1000-step run from the
initial load (restored from a device snapshot before each step, outside the timed region) on
the library's production path: per 50-step period the CV in the cheaper of its two exact
forms (the library's cost rule takes the Fourier form here), the Silverman widths, then
50 x (sort, deposit, Poisson, gather + push + field energy).  All of it runs in libkdepic's
CUDA kernels.

`value` = the in-radius (particle, node) pairs of the run's 1000 deposits and 1000 gathers
divided by the run's device time.  Sub-records of the same line: the O(N^2) pair-sum
CV at the CV-sweep configuration (`cv_pairs`), the 256-realisation ensemble
(`ensemble`), the 10,000-request serving stream (`serve`) and the Sec. II.D schedule
(`ad_schedule`).  `--impl reference` times the FP64 CPU oracle on a bounded sample of the
same workload (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "deposit+gather particle·node pairs/s; CV pairs/s; serve p50/p99 vs plain"
UNIT = "pairs/s"

LANDAU = dict(N=1 << 20, Ng=256, L=4 * math.pi, dt=0.1, period=50, run_steps=1000, n_cand=64, kmin_c=1.0,
              kmax_c=1e4, alpha=0.5, kappa_min=1.0, kappa_max=1e5, seed=0)


def workload_name(w):
    return ("landau_damping N=2^20 Ng=256 dt=0.1, 1000 steps from the initial load, widths every 50 steps "
            "(CV over 64 candidates in [1,1e4], alpha=0.5)")


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock and throttle-reason samples every 50 ms, each stamped on arrival.
    Started before the timed region (the tool takes a moment to start); begin() and end()
    mark the timed region, and stop() keeps the samples that arrived inside it (or, when
    the region is shorter than the interval, the samples nearest to it, and says so)."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 50

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def begin(self):
        self.t0 = time.perf_counter()

    def end(self):
        self.t1 = time.perf_counter()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return self.summarise(self.lines, self.t0, self.t1)

    @staticmethod
    def summarise(lines, t0=None, t1=None):
        rows = []
        for t, ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((t, float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return None
        window = "whole run"
        if t0 is not None and t1 is not None:
            inside = [r for r in rows if t0 <= r[0] <= t1]
            if inside:
                rows, window = inside, "timed region"
            else:  # a region shorter than the interval: the samples on either side of it
                before = [r for r in rows if r[0] < t0][-1:]
                after = [r for r in rows if r[0] > t1][:1]
                if before or after:
                    rows, window = before + after, "nearest to the timed region"
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for nm, val in zip(names, r[3]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median([r[1] for r in rows])), "sm_max_mhz": float(max(r[2] for r in rows)),
                "reasons": sorted(reasons), "samples": len(rows), "window": window}


# ---------------------------------------------------------------------------
# algorithmic work of the CV pair kernel: for every candidate, the unordered
# pairs inside its truncation radius (kernel >= 2^-24 of its peak)
# ---------------------------------------------------------------------------
def cv_inradius_pairs(u_np, cands):
    th = np.sort(u_np.astype(np.float64)) * (2 * math.pi / 2 ** 32)
    N = th.size
    ext = np.concatenate([th, th + 2 * math.pi])
    total = 0
    for k in cands:
        s2 = 24.0 * math.log(2.0) / (2.0 * k)
        if s2 >= 1.0:
            total += N * (N - 1) // 2
            continue
        r = 2.0 * math.asin(math.sqrt(s2))
        # pairs j after i (circularly) within r: with r < pi each unordered pair is
        # counted exactly once, from the particle it follows
        hi = np.searchsorted(ext, th + r, side="right")
        cnt = np.minimum(hi - np.arange(N) - 1, N - 1)
        total += int(cnt.sum())
    return total


def grid_window_pairs(kappa_np, Ng, cut=24.0):
    """(particle, node) pairs inside the truncation radius (kernel >= 2^-cut of its peak) for
    one deposit or one gather: per particle the nodes within r = 2 asin(sqrt(cut ln2 / (2 kappa)))
    of it, 2 r Ng / (2 pi) on average over positions, at most Ng."""
    k = np.asarray(kappa_np, dtype=np.float64)
    s2 = np.minimum(cut * math.log(2.0) / (2.0 * k), 1.0)
    r = 2.0 * np.arcsin(np.sqrt(s2))
    return float(np.minimum(Ng, r * Ng / math.pi).sum())


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except ValueError:
            return {}
    return {}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (the reference arm and the cpu_baseline leg)
# ---------------------------------------------------------------------------
def oracle_sample(n_steps=10, N=1 << 12):
    import kde_inputs as I
    import oracle as O
    w = LANDAU
    O.build()
    u, v = I.landau_load(w["seed"], N, w["L"], 0.05, 1.0)
    x = I.from_fixed(u, w["L"])
    cand = I.log_candidates(w["kmin_c"], w["kmax_c"], w["n_cand"])
    t0 = time.perf_counter()
    O.pic_run(x, v.astype(np.float32), w["L"], w["Ng"], w["dt"], n_steps, kappa=np.ones(N), width_every=w["period"],
              cands=cand, alpha=w["alpha"], kmin=w["kappa_min"], kmax=w["kappa_max"])
    dt = time.perf_counter() - t0
    pairs = 2.0 * N * w["Ng"] * n_steps
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return pairs / dt, dt, cores, "%d particles, Ng=%d, %d PIC steps incl. one CV width update over %d candidates" % (
        N, w["Ng"], n_steps, w["n_cand"])


def run_reference(args, rank, world):
    if rank != 0:
        return
    # each step: one width-update period (CV + 50 PIC steps) of a 2^15-particle sample
    for _ in range(args.warmup):
        oracle_sample(2)
    vals, times = [], []
    for _ in range(args.steps):
        v, dt, cores, sample = oracle_sample(LANDAU["period"], 1 << 15)
        vals.append(v)
        times.append(dt)
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(LANDAU), "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def over_ranks(x, dist, device, op="max"):
    """x reduced over the ranks (the largest time, or the sum of work); x itself without a
    process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def replicas_rate(units_all_ranks, t_ms_slowest):
    """Whole-job throughput of independent replicas: the units of every rank over the slowest
    rank's time."""
    return units_all_ranks / (t_ms_slowest * 1e-3)


def timed(fn, flush, reps):
    """CUDA-event times (ms) of reps calls of fn on the current stream, L2 flushed before each."""
    import torch
    out = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        out.append(a.elapsed_time(b))
    return out


def landau_state(kp, dev, w, seed, max_steps, **kw):
    import torch

    import kde_inputs as I
    N, Ng, L, dt, P = w["N"], w["Ng"], w["L"], w["dt"], w["period"]
    cand = I.log_candidates(w["kmin_c"], w["kmax_c"], w["n_cand"])
    u0, v0 = I.landau_load(seed, N, L, 0.05, 1.0)
    st = kp.PicState(torch.from_numpy(u0.view(np.int32)).to(dev), torch.from_numpy(v0.astype(np.float32)).to(dev),
                     L, Ng, dt, kappa=torch.ones(N, device=dev), ids=torch.arange(N, dtype=torch.int32, device=dev),
                     width_every=P, cand=cand, alpha=w["alpha"], kappa_min=w["kappa_min"], kappa_max=w["kappa_max"],
                     max_steps=max_steps, **kw)
    return st, u0, v0, cand


def cv_pairs_record(kp, ctx, dev, ex2_peak, reps=3):
    """The O(N^2) pair-sum CV of Eq. cv_def at the CV-sweep configuration: N = 2^18 positions
    from 0.7 U + 0.3 vonMises(pi, 20), 64 candidates in [1, 1e4], forced pair sums (the
    production path would take the exact Fourier form).  Definition pairs/s and the exp2
    roofline of the pair kernel."""
    import torch

    import kde_inputs as I
    N, L = 1 << 18, 2 * math.pi
    cand = I.log_candidates(1.0, 1e4, 64)
    u_np = I.cv_sweep_load(0, N)
    u = torch.from_numpy(u_np.view(np.int32)).to(dev)
    loo = torch.empty(N, device=dev)
    ctx.cv(u, L, cand, loo=loo, pairs=True)
    ctx.profile_enable(True)
    t0 = time.perf_counter()
    for _ in range(reps):
        ctx.cv(u, L, cand, loo=loo, pairs=True)
    wall = (time.perf_counter() - t0) / reps
    cv_ms, cv_n = ctx.profile_read("cv_pairs")
    ctx.profile_enable(False)
    alg = cv_inradius_pairs(u_np, cand)
    launch_ms = cv_ms / max(cv_n, 1)
    ach = alg / (launch_ms * 1e-3)
    return {"workload": "CV width sweep: N=2^18 mixture 0.7U+0.3vM(pi,20) on [0,2pi), 64 candidates in [1,1e4], "
                        "O(N^2) pair sums (KDE_CV_PAIRS)",
            "cv_pairs_per_s": 64 * N * (N - 1) / (wall), "unit": "definition pairs/s (64 N (N-1) per call)",
            "ms_per_call": 1e3 * wall, "pair_kernel_ms": launch_ms,
            "roofline": {"bound": "alu", "kernel": "cv_pairs_fast_kernel", "achieved": ach / 1e12,
                         "peak": ex2_peak / 1e12, "unit": "Tex2/s", "frac": ach / ex2_peak,
                         "algorithmic_units_per_launch": alg,
                         "unit_def": "one exp2 per (unordered pair inside the candidate's truncation radius, "
                                     "candidate)"}}


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_1804_11174_gb300 as kp
    from paper_1804_11174_gb300 import _build

    _build.build()
    torch.cuda.set_device(local_rank)
    dev = "cuda:%d" % local_rank
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(dev))

    w = LANDAU
    N, Ng, L, dt, P, RUN = w["N"], w["Ng"], w["L"], w["dt"], w["period"], w["run_steps"]
    ctx = kp.Context(local_rank)
    ctx.reserve(N, Ng, w["n_cand"])
    ctx.set_autotune(not args.no_autotune)  # gather shape and truncation cut tuned on the first step
    # each rank simulates its own realisation (independent replicas, weak scaling).  A bench
    # step is the whole 1000-step run from the initial load: every step repeats it from a
    # snapshot of that load (restored outside the timed region), so the work is the same
    # whatever the number of steps
    st, u0, v0, cand = landau_state(kp, dev, w, w["seed"] + rank, RUN,
                                    cv_spectral=args.cv == "spectral", cv_pairs=args.cv == "pairs")
    snap = st.snapshot()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # 256 MB > 129 MB L2
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()  # before the warm-up: the sampler is running when the timed region starts
    # first warm-up run period by period: the widths in force in each period (set by its
    # first-step update) give the in-radius pair count of its 50 deposits and 50 gathers,
    # at the truncation cut in force (the autotuner's choice for this key, else 2^-24)
    cut, pairs = 24.0, []
    for p in range(RUN // P):
        ctx.pic_step(st, P)
        if p == 0:
            for e in ctx.autotune_table():
                if e["kind"] == "cut_log2" and (e["Ng"], e["log2_N"], e["width_class"]) == (
                        Ng, N.bit_length() - 1, 0):
                    cut = e["value"]
        pairs.append(2.0 * P * grid_window_pairs(st.kappa.cpu().numpy(), Ng, cut))
    energy_ref = st.energy.clone()
    for _ in range(args.warmup - 1):
        st.restore(snap)
        ctx.pic_step(st, RUN)
    torch.cuda.synchronize()

    # ---- the config's run: 20 production width-update periods (CV by the cost rule + Silverman
    #      widths + 50 PIC steps), one pic_step call ----
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.begin()
    ctx.profile_enable(False)  # no events between the kernels (they would serialise the launch overlap);
    #                            this also zeroes the launch counter
    wall0 = time.perf_counter()
    step_ms, repeat_ok = [], True
    for _ in range(args.steps):
        st.restore(snap)
        step_ms += timed(lambda: ctx.pic_step(st, RUN), flush, 1)
        repeat_ok = repeat_ok and bool(torch.equal(st.energy, energy_ref))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks.end()
    _, launches = ctx.profile_read("all")
    # per-kernel durations: CUDA events around every kernel over one more run
    st.restore(snap)
    ctx.profile_enable(True)
    prof_ms = timed(lambda: ctx.pic_step(st, RUN), flush, 1)
    prof = {k: ctx.profile_read(k) for k in ("deposit", "gather", "sort", "poisson", "spectral", "cv_pairs",
                                              "cv_grid", "cv_loo")}
    ctx.profile_enable(False)
    clk = clocks.stop()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_step = over_ranks(float(np.mean(step_ms)), dist, dev, "max")
    pairs_run = float(np.sum(pairs))
    pairs_all = over_ranks(pairs_run, dist, dev, "sum")
    value = replicas_rate(pairs_all, t_step)

    # ---- e2e: the same run through the C ABI from pinned host buffers (pic_step_host: host ->
    #      device copies of u, v, kappa, id, the run, copies back of them and of the histories,
    #      inside the call) ----
    sd = snap[0]
    host = kp.PicState(sd["u"].cpu().pin_memory(), sd["v"].cpu().pin_memory(), L, Ng, dt,
                       kappa=sd["kappa"].cpu().pin_memory(), ids=sd["id"].cpu().pin_memory(), width_every=P,
                       cand=cand, alpha=w["alpha"], kappa_min=w["kappa_min"], kappa_max=w["kappa_max"],
                       max_steps=RUN, cv_spectral=args.cv == "spectral", cv_pairs=args.cv == "pairs")
    hsnap = host.snapshot()
    for _ in range(max(1, min(args.warmup, 2))):
        host.restore(hsnap)
        ctx.pic_step_host(host, RUN)
    e_ms = []
    for _ in range(max(1, min(args.steps, 5))):
        host.restore(hsnap)
        e_ms += timed(lambda: ctx.pic_step_host(host, RUN), flush, 1)
    e_t = over_ranks(float(np.mean(e_ms)), dist, dev, "max")
    n_hist = sum(t is not None for t in (host.energy, host.kappa_star, host.ad_log_p))
    e2e = {"value": replicas_rate(pairs_all, e_t), "unit": UNIT, "ms_per_step": e_t,
           "h2d_bytes_per_step": N * 16, "d2h_bytes_per_step": N * 16 + n_hist * RUN * 8,
           "path": "pic_step_host (C ABI, pinned host buffers; copies inside the call)"}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    ms_p, ops_p = ctx.probe_exp2(1 << 14)
    ex2_peak = ops_p / (ms_p * 1e-3)
    fm_ms, fm_ops = ctx.probe_fma(1 << 14)
    kr = {}
    per_launch = pairs_run / (2.0 * RUN)  # in-radius pairs of one deposit (or one gather), run average
    for name, key in (("deposit_persist_kernel", "deposit"), ("gather2_kernel", "gather")):
        ms_k, n_k = prof[key]
        if n_k:
            ach_k = per_launch / (ms_k / n_k * 1e-3)
            kr[name] = {"bound": "alu", "achieved": ach_k / 1e12, "peak": ex2_peak / 1e12, "unit": "Tex2/s",
                        "frac": ach_k / ex2_peak, "algorithmic_units_per_launch": per_launch,
                        "avg_launch_ms": ms_k / n_k, "launches": n_k,
                        "unit_def": "one exp2 per (particle, node) pair inside the particle's truncation radius"}
    s_ms, s_n = prof["sort"]
    hbm = measured_peaks().get("hbm_gbs") or 6773.2
    if s_n:
        ncounts = Ng * -(-N // 2048)  # (bin, tile) count entries: tiles of 2048 particles
        sort_bytes = N * (20 + 20) + 12 * ncounts
        ach_s = sort_bytes / (s_ms / s_n * 1e-3) / 1e9
        kr["sort_scan+scatter"] = {
            "bound": "hbm", "achieved": ach_s, "peak": hbm, "unit": "GB/s", "frac": ach_s / hbm,
            "algorithmic_bytes_per_launch": sort_bytes, "avg_launch_ms": s_ms / s_n, "launches": s_n,
            "unit_def": "per particle 20 B read and 20 B written by the scatter (u, v, kappa, norm, id); per "
                        "(bin, tile) count entry 12 B (the scan's read and write, and the zeroing of the other "
                        "table); the counts themselves are added by the gather + push of the step before"}
    dom = max(("deposit_persist_kernel", "gather2_kernel"),
              key=lambda k: kr[k]["avg_launch_ms"] * kr[k]["launches"] if k in kr else -1.0)
    roof = dict(kr.get(dom, {}), kernel=dom, traffic=PROFILED_TRAFFIC.get(dom),
                peak_source="measured ex2.approx.ftz.f32 stream on this GPU (kde_probe_exp2)",
                fma_peak_tflops=2.0 * fm_ops / (fm_ms * 1e-3) / 1e12)

    sub = {}
    if not args.quick:
        try:
            sub["cv_pairs"] = cv_pairs_record(kp, ctx, dev, ex2_peak)
        except Exception as e:  # report, do not fail the main line
            sub["cv_pairs"] = {"error": str(e)}
        try:
            sub["ensemble"] = ensemble_record(kp, ctx, dev, args)
        except Exception as e:
            sub["ensemble"] = {"error": str(e)}
        try:
            sub["serve"] = serve_record(kp, args)
        except Exception as e:
            sub["serve"] = {"error": str(e)}
        try:
            sub["ad_schedule"] = ad_record(kp, ctx, dev, args, flush)
        except Exception as e:
            sub["ad_schedule"] = {"error": str(e)}

    try:
        if args.no_cpu_baseline:
            raise RuntimeError("skipped (--no-cpu-baseline)")
        # one width-update period (CV + 50 PIC steps) of a 2^18-particle sample: 10-30 s of CPU work
        cpu_v, cpu_dt, cores, sample = oracle_sample(LANDAU["period"], 1 << 18)
        cpu = {"value": cpu_v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "seconds": cpu_dt}
    except Exception as e:  # the oracle needs gcc; report its absence instead of failing the bench
        cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": "unavailable: %s" % e}

    cv_form = {"auto": "cost rule (exact Fourier form on this load)", "pairs": "O(N^2) pair sums",
               "spectral": "exact Fourier form"}[args.cv]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(w), "N": N, "Ng": Ng, "dt": dt, "pic_steps_per_step": RUN,
                   "width_period": P, "n_cand": w["n_cand"], "cv_form": cv_form,
                   "value_def": "in-radius deposit+gather (particle, node) pairs of the 1000-step run / run time",
                   "l2": "flushed before every timed step (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single",
                   "gather_tile_shape": "default" if args.no_autotune else "autotuned",
                   "truncation_cut_log2": cut,
                   "repeat": "every step restarts from a snapshot of the initial load (restored outside the "
                             "timed region); its energy history equals the first run's bit for bit: %s" % repeat_ok},
        "pairs_per_step": pairs_run,
        "pairs_per_period": pairs,
        "kernel_ms_per_step": {k: v[0] for k, v in prof.items() if v[1]},
        "kernel_timing": "CUDA events around each kernel on the library's stream over one further run right "
                         "after the timed ones (%.3f ms with the events, which serialise the launch overlap)"
                         % float(np.mean(prof_ms)),
        "wall_s": wall,
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": launches,
        "roofline": roof,
        "kernel_rooflines": kr,
        "cpu_baseline": cpu,
    }
    line.update(sub)
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def ad_record(kp, ctx, dev, args, flush):
    """The Landau load with a uniform width under the Sec. II.D schedule: the Anderson-Darling
    test every step, CV (exact Fourier form) when the p-value halves, smoothing rate 0.05."""
    import torch
    w = LANDAU
    P = w["period"]
    st, _, _, cand = landau_state(kp, dev, w, w["seed"], P * 4, cv_spectral=True)
    st4 = kp.PicState(st.u, st.v, w["L"], w["Ng"], w["dt"], kappa_uniform=50.0, cand=cand, max_steps=P * 4,
                      width_ad=True, cv_spectral=True)
    ctx.pic_step(st4, P)
    torch.cuda.synchronize()
    ctx.profile_enable(True)
    a_ms = timed(lambda: ctx.pic_step(st4, P), flush, 2)
    ad_ms, ad_n = ctx.profile_read("ad")
    ctx.profile_enable(False)
    at = float(np.mean(a_ms))
    lp = st4.ad_log_p.cpu().numpy()[:st4.c.step]
    return {"schedule": "Anderson-Darling test every step (Sec. II.D), uniform width, CV by the exact Fourier form",
            "ms_per_step": at, "value": 2.0 * P * w["N"] * w["Ng"] / (at * 1e-3),
            "value_def": "deposit+gather (particle, node) pairs (whole-grid windows) / period time",
            "ad_terms_kernel_ms_per_pic_step": ad_ms / max(ad_n, 1), "optimisations": int(st4.c.n_opt),
            "kappa_final": float(st4.c.kappa_uniform), "log_p_first_last": [float(lp[0]), float(lp[-1])]}


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the kernels, from
# one ncu capture of each on this Landau step (a PIC step after the tuner's runs; the gather
# with its push on a step that is not a call's last); None once a kernel changes after its
# capture
PROFILED_TRAFFIC = {"deposit_persist_kernel": 12666368 + 0, "gather2_kernel": 16898816 + 0}


def run_cv_sweep(args, rank, world, local_rank):
    """The CV-sweep workload: N = 2^18 positions from 0.7 U + 0.3 vonMises(pi, 20) on
    [0, 2 pi), 64 candidates log-spaced in [1, 1e4]; one step = one kde_cv call (the form
    --cv names: pair sums and integral term, or the exact Fourier form, or the cost rule's
    choice; argmin and leave-one-out pass).  value = CV definition pairs/s."""
    import torch

    import kde_inputs as I
    import paper_1804_11174_gb300 as kp
    from paper_1804_11174_gb300 import _build

    _build.build()
    torch.cuda.set_device(local_rank)
    dev = "cuda:%d" % local_rank
    N, L = 1 << 18, 2 * math.pi
    cand = I.log_candidates(1.0, 1e4, 64)
    u_np = I.cv_sweep_load(rank, N)
    u = torch.from_numpy(u_np.view(np.int32)).to(dev)
    ctx = kp.Context(local_rank)
    loo = torch.empty(N, device=dev)
    for _ in range(args.warmup):
        ctx.cv(u, L, cand, loo=loo, pairs=args.cv == "pairs", spectral=args.cv == "spectral")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ms = []
    ctx.profile_enable(True)
    for _ in range(args.steps):
        flush.zero_()
        t0 = time.perf_counter()
        ctx.cv(u, L, cand, loo=loo, pairs=args.cv == "pairs", spectral=args.cv == "spectral")
        ms.append(1e3 * (time.perf_counter() - t0))
    cv_ms, cv_n = ctx.profile_read("cv_pairs")
    _, launches = ctx.profile_read("all")
    ctx.profile_enable(False)
    t = float(np.mean(ms))
    if rank == 0:
        alg = cv_inradius_pairs(u_np, cand)
        ms_p, ops_p = ctx.probe_exp2(1 << 14)
        peak = ops_p / (ms_p * 1e-3)
        ach = alg / (cv_ms / cv_n * 1e-3)
        line = {"metric": METRIC, "value": world * 64 * N * (N - 1) / (t * 1e-3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "cv_sweep N=2^18 mixture 0.7U+0.3vM(pi,20), 64 candidates in [1,1e4]"},
                "gpu_launches": launches,
                "roofline": {"bound": "alu", "kernel": "cv_pairs_fast_kernel", "achieved": ach / 1e12, "peak": peak / 1e12,
                             "unit": "Tex2/s", "frac": ach / peak, "traffic": None,
                             "avg_launch_ms": cv_ms / cv_n}}
        print(json.dumps(line), flush=True)
    ctx.close()


def serve_requests(R, seed=0, nmax_log2=22, cv_nmax_log2=17):
    """The serving stream: kinds cycle deposit / gather / CV (16 scale factors on kappa_i) /
    10-step PIC; N = floor(2^(12 + (nmax-12) U)), log-uniform in [2^12, 2^nmax] (CV requests
    capped at 2^cv_nmax: their pair sums are O(N^2)); Ng log-uniform integer in [64, 4096];
    kappa_i log-uniform in [5, 5e3]; Maxwellian v_th = 1; uniform positions.  Requests are
    slices of one shared host pool held in page-locked memory."""
    import torch

    import kde_inputs as I
    pool = 1 << nmax_log2
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    u = pin((I.splitmix64(seed, I.STREAM_X, pool) >> np.uint64(32)).astype(np.uint32))
    kap = pin(I.log_uniform(seed, I.STREAM_KAPPA, pool, 5.0, 5e3).astype(np.float32))
    v = pin(I.maxwellian(seed, pool, 1.0).astype(np.float32))
    U = I.uniforms(seed, I.STREAM_REQ, 3 * R)
    scales = 10.0 ** ((np.arange(16) - 8) / 8.0)
    reqs = []
    for q in range(R):
        kind = 1 + q % 4
        top = cv_nmax_log2 if kind == 3 else nmax_log2
        N = int(2 ** (12 + (top - 12) * U[3 * q]))
        Ng = int(round(64 * 64 ** U[3 * q + 1]))
        off = int(U[3 * q + 2] * (pool - N))
        r = dict(kind=kind, N=N, Ng=Ng, u=u[off:off + N], kappa=kap[off:off + N])
        if kind == 2:
            r["field"] = np.sin(2 * math.pi * np.arange(Ng) / Ng).astype(np.float32)
        if kind == 3:
            r["cand"] = scales
        if kind == 4:
            r["v"] = v[off:off + N]
        reqs.append(r)
    return reqs


def serve_stream(kp, reqs, n_slots, arrivals, outs):
    """Submit each request at its arrival time (seconds from start) and return latencies (ms)
    and the makespan (s).  outs: preallocated page-locked output buffers per request."""
    srv = kp.Server(0, n_slots=n_slots, hbm_budget_bytes=100 << 30)
    L = 4 * math.pi
    tickets = []
    t0 = time.perf_counter()
    for r, ta, (out, out64) in zip(reqs, arrivals, outs):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        tickets.append(srv.submit(r["kind"], r["u"], L, Ng=r["Ng"], kappa=r["kappa"], v=r.get("v"),
                                  field=r.get("field"), cand=r.get("cand"), n_steps=10 if r["kind"] == 4 else 0,
                                  dt=0.1, out=out, out64=out64))
    lat = np.array([srv.wait(t)[0] for t in tickets])
    span = time.perf_counter() - t0
    srv.close()
    return lat, span


def serve_outputs(reqs):
    import torch
    pin = lambda n, dt: torch.empty(n, dtype=dt).pin_memory().numpy()
    outs = []
    for r in reqs:
        out = pin(r["Ng"] if r["kind"] == 1 else r["N"], torch.float32) if r["kind"] in (1, 2, 4) else None
        out64 = pin(16 if r["kind"] == 3 else 10, torch.float64) if r["kind"] in (3, 4) else None
        outs.append((out, out64))
    return outs


def serve_record(kp, args):
    """Continuous batching (args.slots slots) against the plain form (one slot: one request at a
    time) on the same stream of args.requests requests: saturated throughput (everything
    submitted at t = 0) and p50/p99 latency under Poisson arrivals at 0.9x the plain
    throughput, each pair run args.serve_repeats times."""
    import kde_inputs as I
    R = args.requests
    t_build = time.perf_counter()
    reqs = serve_requests(R, nmax_log2=args.serve_nmax_log2, cv_nmax_log2=args.serve_cv_nmax_log2)
    outs = serve_outputs(reqs)
    t_build = time.perf_counter() - t_build
    warm = serve_requests(32, seed=99, nmax_log2=args.serve_nmax_log2, cv_nmax_log2=args.serve_cv_nmax_log2)
    wouts = serve_outputs(warm)
    serve_stream(kp, warm, args.slots, np.zeros(len(warm)), wouts)
    serve_stream(kp, warm, 1, np.zeros(len(warm)), wouts)
    pct = lambda a, q: float(np.percentile(a, q))
    runs = []
    for rep in range(args.serve_repeats):
        _, span_p = serve_stream(kp, reqs, 1, np.zeros(R), outs)
        _, span_b = serve_stream(kp, reqs, args.slots, np.zeros(R), outs)
        mu_plain = R / span_p
        gaps = -np.log(1.0 - I.uniforms(7 + rep, 7, R)) / (0.9 * mu_plain)
        arr = np.cumsum(gaps) - gaps[0]
        lat_p, _ = serve_stream(kp, reqs, 1, arr, outs)
        lat_b, _ = serve_stream(kp, reqs, args.slots, arr, outs)
        runs.append({"saturated_rps": {"batched": R / span_b, "plain": mu_plain},
                     "poisson_rate_rps": 0.9 * mu_plain,
                     "batched": {"p50_ms": pct(lat_b, 50), "p99_ms": pct(lat_b, 99)},
                     "plain": {"p50_ms": pct(lat_p, 50), "p99_ms": pct(lat_p, 99)}})
    Ns = np.array([r["N"] for r in reqs])
    return {"workload": "serving: %d requests cycling deposit / gather / CV (16 scales of kappa_i) / 10-step "
                        "pic_step; N log-uniform in [2^12, 2^%d] (CV requests capped at 2^%d); Ng log-uniform in "
                        "[64, 4096]; kappa_i log-uniform in [5, 5e3]; Maxwellian v; page-locked host buffers; "
                        "HBM budget 100 GB; batched = %d slots, plain = 1 slot"
                        % (R, args.serve_nmax_log2, args.serve_cv_nmax_log2, args.slots),
            "requests": R, "particles_total": int(Ns.sum()), "largest_N": int(Ns.max()),
            "runs": runs,
            "batched_over_plain_rps": [r["saturated_rps"]["batched"] / r["saturated_rps"]["plain"] for r in runs],
            "p99_batched_over_plain": [r["batched"]["p99_ms"] / r["plain"]["p99_ms"] for r in runs],
            "host_build_s": t_build}


def run_serve(args, rank, world, local_rank):
    import paper_1804_11174_gb300 as kp
    from paper_1804_11174_gb300 import _build
    _build.build()
    if rank != 0:
        return
    rec = serve_record(kp, args)
    r0 = rec["runs"][0]
    line = {"metric": METRIC, "value": r0["saturated_rps"]["batched"], "unit": "requests/s", "n_gpus": 1,
            "steps": 1, "warmup": 1, "ms_per_step": 1e3 * args.requests / r0["saturated_rps"]["batched"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": rec["workload"]}, "serve": rec}
    print(json.dumps(line), flush=True)


def ensemble_record(kp, ctx, dev, args):
    """Ensemble: R independent Landau realisations (seeds 0..R-1, alpha = 0.05, v_th = 1,
    dt = 0.1), N log-uniform in [2^14, 2^20], Ng cycling {128, 256, 512, 1024}, one uniform width
    per realisation chosen at t = 0 by the CV (exact Fourier form) over 16 candidates in
    [1, 1e3].  One step = one replay of the captured graph over all realisations; compared with
    the same launches issued directly and with the plain form (pic_step per realisation, one
    after another, on one stream; a 32-realisation sample scaled by particle count)."""
    import torch

    import kde_inputs as I
    R = args.realisations
    L = 4 * math.pi
    Ns, Ngs = I.ensemble_sizes(R)
    us, vs = [], []
    t_build = time.perf_counter()
    for r in range(R):
        q = I.uniforms(r, I.STREAM_X, int(Ns[r]))
        us.append(I.to_fixed(I.inverse_cdf_cosine(q, L, 0.05), L))
        vs.append(I.maxwellian(r, int(Ns[r]), 1.0).astype(np.float32))
    t_build = time.perf_counter() - t_build
    cand = I.log_candidates(1.0, 1e3, 16)
    kap = []
    for r in range(R):
        _, am, _ = ctx.cv(torch.from_numpy(us[r].view(np.int32)).to(dev), L, cand, spectral=True)
        kap.append(float(cand[am]))
    u = torch.from_numpy(np.concatenate(us).view(np.int32)).to(dev)
    v = torch.from_numpy(np.concatenate(vs)).to(dev)
    ens = kp.Ensemble(ctx, Ns, Ngs, kap, L, 0.1, u, v)
    mise = ens.mise(0.05, 1).cpu().numpy()
    steps = args.ens_steps
    en = torch.zeros(R * steps, dtype=torch.float64, device=dev)
    ens.run(1, None, use_graph=True)
    ens.run(steps, en, use_graph=True)  # captures the step for this (energy, steps) pair
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    t_graph = timed(lambda: ens.run(steps, en, use_graph=True), flush, 2)
    t_launch = timed(lambda: ens.run(steps, en, use_graph=False), flush, 1)
    t_graph, t_launch = min(t_graph) / steps, t_launch[0] / steps
    sample = min(R, 32)
    sts = [kp.PicState(torch.from_numpy(us[r].view(np.int32)).to(dev), torch.from_numpy(vs[r]).to(dev), L,
                       int(Ngs[r]), 0.1, kappa_uniform=kap[r]) for r in range(sample)]
    for s_ in sts:
        ctx.pic_step(s_, 1)
    torch.cuda.synchronize()

    def plain():
        for _ in range(3):
            for s_ in sts:
                ctx.pic_step(s_, 1)
    frac = float(np.sum(Ns[:sample])) / float(np.sum(Ns))
    t_plain = timed(plain, flush, 1)[0] / 3 / frac
    ens.close()
    # the autotuner's choice per key of the realisations (grid size, log2 N, width class)
    keys = {}
    for r in range(R):
        wc = min(255, max(1, int(4.0 * math.log2(kap[r]) + 128.0)))
        keys[(int(Ngs[r]), int(Ns[r]).bit_length() - 1, wc)] = kap[r]
    tuned = {}
    for e in ctx.autotune_table():
        kk = (e["Ng"], e["log2_N"], e["width_class"])
        if kk in keys:
            tuned.setdefault(kk, {"Ng": kk[0], "log2_N": kk[1], "kappa": keys[kk]})[e["kind"]] = e["value"]
    cut_hist = {}
    for t in tuned.values():
        if "cut_log2" in t:
            cut_hist[str(t["cut_log2"])] = cut_hist.get(str(t["cut_log2"]), 0) + 1
    Ntot = float(np.sum(Ns))
    return {"workload": "ensemble of %d Landau realisations, N log-uniform in [2^14, 2^20] (total %d), Ng in "
                        "{128,256,512,1024}, one CUDA graph per step" % (R, int(Ntot)),
            "particles": int(Ntot), "ms_per_step_graph": t_graph, "ms_per_step_launches": t_launch,
            "ms_per_step_plain_per_realisation": t_plain,
            "particle_steps_per_s_graph": Ntot / (t_graph * 1e-3),
            "particle_steps_per_s_plain": Ntot / (t_plain * 1e-3),
            "graph_over_plain": t_plain / t_graph,
            "pairs_per_s_graph_definition": 2.0 * float(np.sum(Ns * Ngs)) / (t_graph * 1e-3),
            "mise_t0": {"mean": float(np.mean(mise)), "min": float(np.min(mise)), "max": float(np.max(mise))},
            "kappa_star": {"min": float(np.min(kap)), "max": float(np.max(kap))},
            "autotune": {"keys": len(keys), "tuned": sorted(tuned.values(), key=lambda t: (t["Ng"], t["log2_N"],
                                                                                          t["kappa"])),
                         "cut_log2_histogram": cut_hist},
            "l2": "inputs larger than L2 (%.0f MB of particle state)" % (Ntot * 8 / 1e6),
            "host_build_s": t_build}


def run_ensemble(args, rank, world, local_rank):
    import torch

    import paper_1804_11174_gb300 as kp
    from paper_1804_11174_gb300 import _build
    _build.build()
    torch.cuda.set_device(local_rank)
    dev = "cuda:%d" % local_rank
    ctx = kp.Context(local_rank)
    ctx.set_autotune(not args.no_autotune)  # the lanes tune their gathers in the first (uncaptured) step
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    rec = ensemble_record(kp, ctx, dev, args)
    clk = clocks.stop()
    line = {"metric": METRIC, "value": rec["pairs_per_s_graph_definition"], "unit": UNIT, "n_gpus": 1,
            "steps": args.ens_steps, "warmup": 1, "ms_per_step": rec["ms_per_step_graph"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": rec["workload"], "l2": rec["l2"]}, "ensemble": rec, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def run_shapes(args, rank, world, local_rank):
    """Shape comparison of Sec. IV (Fig. compare_high_order) on the GPU: the density
    1 + 0.02 cos x on [0, 2 pi), N = 2^19 random particles, Ng = 512; MISE (probability-density
    units, averaged over independent loads) and time per estimate for (a-d) B-spline shapes of
    degree 1, 2, 3, 5 at width dx, (e) von Mises with sigma = 2 dx, (f) CIC with the CV width,
    (g) von Mises with the CV width, (h) von Mises with Silverman widths around it."""
    import torch

    import kde_inputs as I
    import paper_1804_11174_gb300 as kp
    from paper_1804_11174_gb300 import _build
    _build.build()
    torch.cuda.set_device(local_rank)
    dev = "cuda:%d" % local_rank
    L, Ng, N, alpha = 2 * math.pi, 512, 1 << 19, 0.02
    R = args.loads
    dx = L / Ng
    truth = 1.0 + alpha * np.cos(2 * math.pi * np.arange(Ng) / Ng)
    ctx = kp.Context(local_rank)
    kap_cand = I.log_candidates(1.0, 1e4, 64)
    h_cand = dx * 2.0 ** (np.arange(28) / 4.0)  # dx .. 104 dx (the CV needs 4 h < L)
    kap_e = 1.0 / (2 * dx) ** 2  # sigma = 2 dx (theta = x on [0, 2 pi))

    def est(method, du):
        if method.startswith("bspline"):
            return ctx.deposit_bspline(du, Ng, L, int(method[-1]), dx), None
        if method == "vm_2dx":
            return ctx.deposit(du, Ng, L, kappa_uniform=kap_e), kap_e
        if method == "cic_cv":
            cv, am = ctx.cv_cic(du, L, h_cand)
            return ctx.deposit_bspline(du, Ng, L, 1, float(h_cand[am])), float(h_cand[am])
        _, am, loo = ctx.cv(du, L, kap_cand, spectral=True, want_loo=(method == "vm_adaptive"))
        ks = float(kap_cand[am])
        if method == "vm_cv":
            return ctx.deposit(du, Ng, L, kappa_uniform=ks), ks
        kap = ctx.adapt_widths(loo, L, ks, 0.5, 1.0, 1e6)
        return ctx.deposit(du, Ng, L, kappa=kap), ks

    methods = ["bspline1", "bspline2", "bspline3", "bspline5", "vm_2dx", "cic_cv", "vm_cv", "vm_adaptive"]
    paper = {"bspline1": 2.28031e-3, "bspline2": 1.90144e-3, "bspline3": 1.14667e-3, "bspline5": 0.74505e-3,
             "vm_2dx": 0.43698e-3, "cic_cv": 0.17233e-3, "vm_cv": 0.15423e-3, "vm_adaptive": 0.13063e-3}
    loads = [torch.from_numpy(I.to_fixed(I.random_positions(r, N, L, alpha), L).view(np.int32)).to(dev)
             for r in range(R)]
    for m in methods:  # warm-up (tables, workspace)
        est(m, loads[0])
    torch.cuda.synchronize()
    table = {}
    for m in methods:
        mise, widths, ms = [], [], []
        for du in loads:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rho, w = est(m, du)
            torch.cuda.synchronize()
            ms.append(1e3 * (time.perf_counter() - t0))
            d = rho.double().cpu().numpy() - truth
            mise.append(float(np.sum(d * d) * dx) / L ** 2)  # density -> probability density: / L
            widths.append(w)
        table[m] = {"mise_pdf": float(np.mean(mise)), "mise_sd": float(np.std(mise, ddof=1)),
                    "ms_per_estimate": float(np.median(ms)), "paper_mise": paper[m],
                    "width": None if widths[0] is None else float(np.median(widths))}
    t_cic = table["bspline1"]["ms_per_estimate"]
    line = {"metric": METRIC, "value": N * Ng / (t_cic * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": R,
            "warmup": 1, "ms_per_step": t_cic, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "shape comparison: 1 + 0.02 cos x on [0, 2pi), N = 2^19 random, Ng = 512, "
                                   "%d independent loads" % R},
            "mise": table,
            "note": "MISE in probability-density units (density / 2pi), averaged over the loads; width = kappa "
                    "(von Mises) or h (CIC, x units); paper_mise is the paper's single-run value, context only"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def landau_theory(vth, k=1.0, factor=1.0):
    """Damping rate (Im omega) of the kinetic Langmuir root, 1 + F^2/(k v_th)^2 (1 + z Z(z)) = 0,
    z = omega/(sqrt 2 k v_th), with the deposit/gather smoothing factor F of mode k (1: none)."""
    import scipy.special as sp
    a2 = (factor / (k * vth)) ** 2

    def D(w):
        z = w / (math.sqrt(2.0) * k * vth)
        return 1.0 + a2 * (1.0 + z * 1j * math.sqrt(math.pi) * sp.wofz(z))

    # Newton's method on D from Bohm-Gross estimates with several damping guesses; the least
    # damped root that converges is the Landau root
    best = None
    with np.errstate(all="ignore"):
        for gi in (0.01, 0.1, 0.3, 0.6):
            w = complex(math.sqrt(factor ** 2 + 3.0 * (k * vth) ** 2), -gi)
            for _ in range(200):
                h = 1e-7
                dD = (D(w + h) - D(w - h)) / (2 * h)
                if not np.isfinite(dD) or dD == 0:
                    break
                dw = D(w) / dD
                w -= dw
                if abs(dw) < 1e-13:
                    break
            if np.isfinite(w) and abs(D(w)) < 1e-9 and w.real > 0 and (best is None or w.imag > best.imag):
                best = w
    return best.imag if best is not None else float("nan")


def run_landau_stats(args, rank, world, local_rank):
    """Ensemble statistics of Sec. III.B on the GPU: Landau damping with k = 1 (L = 2 pi),
    perturbation 0.02 cos x, N = 2^15, Ng = 256, dt = 0.01, 1500 steps, for thermal velocities
    0.20 .. 0.45; for each, the same 30 loads (common random numbers) advanced by standard PIC
    (CIC) and by the von Mises KDE (width by CV at t = 0, and sigma = 2 dx), each arm one
    ensemble with one captured graph per step; per load the amplitude damping rate from the
    first two peaks of ln W; mean error against the kinetic root (plain, and with the arm's
    own smoothing of mode 1), t statistics, and the paired CRN comparison."""
    import scipy.special as sps
    import torch

    import kde_inputs as I
    import paper_1804_11174_gb300 as kp
    from paper_1804_11174_gb300 import _build
    _build.build()
    torch.cuda.set_device(local_rank)
    dev = "cuda:%d" % local_rank
    L, Ng, N, dt, steps, R = 2 * math.pi, 256, 1 << 15, 0.01, args.stat_steps, args.ens_size
    dx = L / Ng
    ctx = kp.Context(local_rank)
    cand = I.log_candidates(1.0, 1e3, 16)
    kap_2dx = 1.0 / (2 * dx) ** 2
    cic_factor = (math.sin(dx / 2) / (dx / 2)) ** 2
    out = {}
    t_total = 0.0
    for vth in (0.20, 0.25, 0.30, 0.35, 0.40, 0.45):
        loads = [I.landau_load(1000 * int(round(vth * 100)) + r, N, L, 0.02, vth) for r in range(R)]
        u0 = np.concatenate([a for a, _ in loads])
        v0 = np.concatenate([b.astype(np.float32) for _, b in loads])
        kcv = []
        for a, _ in loads:
            _, am, _ = ctx.cv(torch.from_numpy(a.view(np.int32)).to(dev), L, cand, spectral=True)
            kcv.append(float(cand[am]))
        arms = {"pic_cic": (0, [kap_2dx] * R, [cic_factor] * R),
                "kde_cv_width": (None, kcv, [float(sps.ive(1, k) / sps.ive(0, k)) for k in kcv]),
                "kde_sigma_2dx": (None, [kap_2dx] * R, [float(sps.ive(1, kap_2dx) / sps.ive(0, kap_2dx))] * R)}
        g_plain = landau_theory(vth)
        res = {"theory_plain": g_plain}
        rates = {}
        for name, (shape, kaps, fac) in arms.items():
            du = torch.from_numpy(u0.view(np.int32)).to(dev)
            dv = torch.from_numpy(v0).to(dev)
            ens = kp.Ensemble(ctx, [N] * R, [Ng] * R, kaps, L, dt, du, dv)
            if shape == 0:
                ens.set_shape(1)
            en = torch.zeros(R * steps, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ens.run(steps, en, use_graph=True)
            torch.cuda.synchronize()
            t_total += time.perf_counter() - t0
            W = en.cpu().numpy().reshape(R, steps)
            ens.close()
            g = []
            for r in range(R):
                try:
                    g.append(kp.damping_rate(W[r], dt))
                except kp.KdeError:
                    g.append(float("nan"))
            g = np.array(g)
            ok = np.isfinite(g)
            gs = np.array([landau_theory(vth, factor=f) for f in fac])
            ok_own = ok & np.isfinite(gs)
            e_plain, e_own = g - g_plain, g - gs
            n_ok = int(ok.sum())

            def tstat(e):
                m = np.isfinite(e)
                n = int(m.sum())
                if n < 2:
                    return None, None, None
                sd = float(np.std(e[m], ddof=1))
                return float(np.mean(e[m])), sd, float(np.mean(e[m]) / (sd / math.sqrt(n)))

            m1, s1, t1 = tstat(e_plain)
            m2, s2, t2 = tstat(np.where(ok_own, e_own, np.nan)) if ok_own.sum() > 1 else (None, None, None)
            rates[name] = g
            res[name] = {"mean_rate": float(np.mean(g[ok])), "sd_rate": s1, "loads_with_two_peaks": n_ok,
                         "error_vs_plain_theory": m1, "t_vs_plain_theory": t1,
                         "theory_with_own_smoothing_mean": float(np.nanmean(gs)) if np.isfinite(gs).any() else None,
                         "error_vs_own_theory": m2, "t_vs_own_theory": t2,
                         "kappa_median": float(np.median(kaps)) if shape is None else None}
        # paired (common random numbers): the CIC arm's absolute error minus the KDE arm's, per load
        for kde in ("kde_cv_width", "kde_sigma_2dx"):
            d = np.abs(rates["pic_cic"] - g_plain) - np.abs(rates[kde] - g_plain)
            ok = np.isfinite(d)
            sd = float(np.std(d[ok], ddof=1))
            res["paired_abs_error_pic_minus_" + kde] = {"mean": float(np.mean(d[ok])), "sd": sd,
                                                        "t": float(np.mean(d[ok]) / (sd / math.sqrt(ok.sum())))}
        out["%.2f" % vth] = res
    particle_steps = 6 * 3 * R * N * steps
    line = {"metric": METRIC, "value": particle_steps / t_total, "unit": "particle-steps/s", "n_gpus": 1,
            "steps": steps, "warmup": 0, "ms_per_step": 1e3 * t_total / (6 * 3 * steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "Landau ensemble statistics: k = 1, 0.02 cos x, N = 2^15, Ng = 256, dt = 0.01, "
                                   "%d steps, %d common-random-number loads per v_th, v_th 0.20..0.45; arms: CIC "
                                   "standard PIC, von Mises at the CV width, von Mises at sigma = 2 dx" % (steps, R)},
            "by_vth": out}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="landau", choices=["landau", "cv_sweep", "serve", "ensemble", "shapes",
                                                            "landau_stats"])
    ap.add_argument("--ens-size", type=int, default=30, help="landau_stats: loads per thermal velocity")
    ap.add_argument("--stat-steps", type=int, default=1500, help="landau_stats: PIC steps per run")
    ap.add_argument("--realisations", type=int, default=256, help="ensemble: realisations")
    ap.add_argument("--loads", type=int, default=8, help="shapes: independent particle loads")
    ap.add_argument("--requests", type=int, default=10000, help="serving: requests in the stream")
    ap.add_argument("--slots", type=int, default=8, help="serving: slots of the batched server")
    ap.add_argument("--serve-repeats", type=int, default=2, help="serving: repeats of each comparison")
    ap.add_argument("--serve-nmax-log2", type=int, default=22, help="serving: largest request size (log2 N)")
    ap.add_argument("--serve-cv-nmax-log2", type=int, default=17, help="serving: largest CV request (log2 N)")
    ap.add_argument("--ens-steps", type=int, default=20, help="ensemble: timed steps per replay")
    ap.add_argument("--quick", action="store_true", help="default line without the sub-records")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle's timed sample (profiling runs)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the gather's default tile shape")
    ap.add_argument("--cv", default="auto", choices=["auto", "pairs", "spectral"],
                    help="CV evaluation (the Landau width schedule and the cv_sweep workload): the library's "
                         "cost rule (auto), O(N^2) pair sums or the exact Fourier form")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "cv_sweep":
        run_cv_sweep(args, rank, world, local_rank)
    elif args.workload == "serve":
        run_serve(args, rank, world, local_rank)
    elif args.workload == "ensemble":
        run_ensemble(args, rank, world, local_rank)
    elif args.workload == "shapes":
        run_shapes(args, rank, world, local_rank)
    elif args.workload == "landau_stats":
        run_landau_stats(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
