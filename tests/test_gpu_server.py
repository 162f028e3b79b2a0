"""The request server (continuous batching): every result is bitwise the same alone and in
the mix, and matches the direct entry points and the oracle."""
import math

import numpy as np
import pytest
import torch

import kde_inputs as I
from conftest import rel_l2, to_dev, to_dev_u

pytestmark = pytest.mark.gpu
L = 4 * math.pi


def make_requests(seed, count, nmax_log2=16):
    reqs = []
    kinds = [1, 2, 3, 4]
    for q in range(count):
        s = seed * 1000 + q
        N = int(2 ** (10 + (nmax_log2 - 10) * I.uniforms(s, 20, 1)[0]))
        Ng = int(64 * (64 ** I.uniforms(s, 21, 1)[0]))
        u, v = I.landau_load(s, N, L, 0.05, 1.0)
        kap = I.log_uniform(s, I.STREAM_KAPPA, N, 5.0, 5e3).astype(np.float32)
        kind = kinds[q % 4]
        r = dict(kind=kind, u=u, Ng=Ng, kappa=kap, v=v.astype(np.float32))
        if kind == 2:
            r["field"] = np.sin(2 * math.pi * np.arange(Ng) / Ng).astype(np.float32)
        if kind == 3:
            r["cand"] = 10.0 ** ((np.arange(8) - 4) / 4.0)
        reqs.append(r)
    return reqs


def run(server, reqs):
    outs, tickets = [], []
    for r in reqs:
        N = r["u"].size
        kind = r["kind"]
        out = np.full(r["Ng"] if kind == 1 else N, np.nan, dtype=np.float32) if kind in (1, 2, 4) else None
        out64 = np.full(8 if kind == 3 else 5, np.nan) if kind in (3, 4) else None
        t = server.submit(kind, r["u"], L, Ng=r["Ng"], kappa=r["kappa"], v=r.get("v"), field=r.get("field"),
                          cand=r.get("cand"), n_steps=5 if kind == 4 else 0, dt=0.1, out=out, out64=out64)
        tickets.append(t)
        outs.append((out, out64))
    res = []
    for t, (out, out64) in zip(tickets, outs):
        lat, svc, am = server.wait(t)
        assert lat >= svc >= 0
        res.append((out, out64, am))
    return res


def test_alone_equals_in_the_mix(kp):
    reqs = make_requests(1, 24)
    alone = kp.Server(0, n_slots=1)
    ref = [run(alone, [r])[0] for r in reqs]  # one at a time
    alone.close()
    mixed = kp.Server(0, n_slots=6)
    got = run(mixed, reqs)  # all submitted together, six slots
    mixed.close()
    for (a, a64, am), (b, b64, bm) in zip(ref, got):
        if a is not None:
            assert np.array_equal(a, b)
        if a64 is not None:
            assert np.array_equal(a64, b64)
        assert am == bm


def test_server_matches_direct_calls_and_oracle(kp, ctx, oracle):
    reqs = make_requests(2, 4, nmax_log2=12)
    srv = kp.Server(0, n_slots=2)
    res = run(srv, reqs)
    srv.close()
    dep, gat, cv, pic = reqs
    x = I.from_fixed(dep["u"], L)
    assert rel_l2(res[0][0], oracle.deposit(x, dep["Ng"], L, kappa=dep["kappa"].astype(np.float64))) <= 1e-5
    direct = ctx.deposit(to_dev_u(dep["u"]), dep["Ng"], L, kappa=to_dev(dep["kappa"])).cpu().numpy()
    assert np.array_equal(direct, res[0][0])
    xg = I.from_fixed(gat["u"], L)
    assert rel_l2(res[1][0], oracle.gather(xg, gat["field"], L, kappa=gat["kappa"].astype(np.float64))) <= 1e-5
    xc = I.from_fixed(cv["u"], L)
    ref = np.array([oracle.cv_dense(xc, L, kappa=s * cv["kappa"].astype(np.float64))[0] for s in cv["cand"]])
    assert np.max(np.abs(res[2][1] - ref)) <= 2e-6 * np.max(np.abs(ref))
    xp = I.from_fixed(pic["u"], L)
    r = oracle.pic_run(xp, pic["v"], L, pic["Ng"], 0.1, 5, kappa=pic["kappa"].astype(np.float64))
    np.testing.assert_allclose(res[3][1], r["energy"], rtol=1e-4)


def test_server_rejects_bad_requests(kp):
    srv = kp.Server(0, n_slots=1, hbm_budget_bytes=1 << 20)
    u = np.arange(1000, dtype=np.uint32)
    with pytest.raises(kp.KdeError):   # larger than the whole budget
        srv.submit(1, u, L, Ng=64, kappa_uniform=5.0, out=np.zeros(64, np.float32))
    with pytest.raises(kp.KdeError):   # missing output
        srv.submit(1, u[:10], L, Ng=64, kappa_uniform=5.0)
    srv.close()


def _pic_request(seed, N, Ng, steps):
    u, v = I.landau_load(seed, N, L, 0.05, 1.0)
    return dict(u=u, v=v.astype(np.float32), Ng=Ng, steps=steps)


def test_work_of_two_slots_overlaps_on_device(kp):
    # two PIC requests of many small launches on two slots: their device-clock intervals
    # (events on each slot's stream around the request) intersect, i.e. the two streams'
    # kernels run interleaved rather than one request after the other
    srv = kp.Server(0, n_slots=2)
    try:
        reqs = [_pic_request(40 + k, 1 << 13, 128, 300) for k in range(2)]
        tickets = []
        for r in reqs:
            out64 = np.zeros(r["steps"])
            tickets.append((srv.submit(4, r["u"], L, Ng=r["Ng"], kappa_uniform=50.0, v=r["v"], n_steps=r["steps"],
                                       dt=0.1, out64=out64), out64))
        iv = []
        for t, out64 in tickets:
            _, _, _, (a, b) = srv.wait(t, times=True)
            assert 0 <= a < b and np.all(np.isfinite(out64))
            iv.append((a, b))
        overlap = min(iv[0][1], iv[1][1]) - max(iv[0][0], iv[1][0])
        print("device intervals (ms): %s, overlap %.3f ms" % (iv, overlap))
        assert overlap > 0.25 * min(b - a for a, b in iv)
    finally:
        srv.close()


def test_budget_accounting_holds_with_retained_workspaces(kp):
    # a budget that holds about two requests' buffers plus workspace: all requests are
    # served, the committed total never passed the budget at an admission, idle slots'
    # workspaces were released to make room, and results equal a one-slot run
    budget = 96 << 20
    reqs = make_requests(7, 16, nmax_log2=17)
    one = kp.Server(0, n_slots=1, hbm_budget_bytes=budget)
    ref = run(one, reqs)
    one.close()
    srv = kp.Server(0, n_slots=4, hbm_budget_bytes=budget)
    try:
        got = run(srv, reqs)
        st = srv.stats()
        print("server stats:", st)
        assert st["served"] == len(reqs) and st["queued"] == 0
        assert st["committed_peak"] <= budget
        assert st["committed"] == st["held"]            # no request buffers outstanding
    finally:
        srv.close()
    for (a, a64, am), (b, b64, bm) in zip(ref, got):
        if a is not None:
            assert np.array_equal(a, b)
        if a64 is not None:
            assert np.array_equal(a64, b64)
        assert am == bm


def test_cancel_queued_request(kp):
    srv = kp.Server(0, n_slots=1)
    try:
        big = _pic_request(50, 1 << 16, 256, 400)
        out_big = np.zeros(400)
        t_big = srv.submit(4, big["u"], L, Ng=256, kappa_uniform=30.0, v=big["v"], n_steps=400, dt=0.1,
                           out64=out_big)
        small = [make_requests(9, 4, nmax_log2=12)[k] for k in range(4)]
        ts = [srv.submit(1, r["u"], L, Ng=r["Ng"], kappa=r["kappa"], out=np.zeros(r["Ng"], np.float32))
              for r in small]
        assert srv.cancel(ts[2]) == 0                  # still queued behind the long request
        with pytest.raises(kp.KdeError) as e:
            srv.wait(ts[2])
        assert e.value.code == 6                       # KDE_ECANCELED
        srv.wait(t_big)
        assert srv.cancel(ts[0]) in (0, 7)             # may already be running or done
        for k in (0, 1, 3):
            try:
                srv.wait(ts[k])
            except kp.KdeError as ex:
                assert k == 0 and ex.code == 6
        assert np.all(np.isfinite(out_big))
        assert srv.cancel(123456789) == 1              # unknown ticket
    finally:
        srv.close()


def test_failed_request_leaves_the_server_serving(kp):
    # a request whose widths are out of range fails on the device (status word, no
    # fault); the requests around it are served and correct
    srv = kp.Server(0, n_slots=2)
    try:
        reqs = make_requests(11, 6, nmax_log2=13)
        bad = dict(reqs[0])
        bad["kappa"] = bad["kappa"].copy()
        bad["kappa"][5] = -1.0
        outs, tickets = [], []
        for r in [reqs[0], bad, reqs[4]]:
            out = np.zeros(r["Ng"], np.float32)
            tickets.append(srv.submit(1, r["u"], L, Ng=r["Ng"], kappa=r["kappa"], out=out))
            outs.append(out)
        srv.wait(tickets[0])
        with pytest.raises(kp.KdeError) as e:
            srv.wait(tickets[1])
        assert e.value.code == 4                       # KDE_EDEVICE: reported, not a fault
        srv.wait(tickets[2])
        alone = kp.Server(0, n_slots=1)
        ref = run(alone, [reqs[0], reqs[4]])
        alone.close()
        assert np.array_equal(outs[0], ref[0][0]) and np.array_equal(outs[2], ref[1][0])
    finally:
        srv.close()
