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
