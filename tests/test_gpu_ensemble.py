"""The ensemble runtime (realisations spread over lanes, one captured CUDA graph per step)
against per-realisation pic_step runs (bitwise: the same kernels on the same states) and the
oracle's MISE."""
import math

import numpy as np
import pytest
import torch

import kde_inputs as I
from conftest import to_dev, to_dev_u

pytestmark = pytest.mark.gpu
L = 4 * math.pi
DEV = "cuda:0"


def loads(Ns, seed0=0):
    us, vs = [], []
    for r, N in enumerate(Ns):
        u, v = I.landau_load(seed0 + r, N, L, 0.05, 1.0)
        us.append(u)
        vs.append(v.astype(np.float32))
    return us, vs


@pytest.mark.parametrize("cut", [0.0, 20.0, 18.0, "tuned"])
def test_ensemble_equals_pic_step_bitwise(ctx, kp, cut):
    # under each truncation choice (the default 2^-24, fixed cuts, and the autotuner's
    # per-key choice, which the lanes share) the ensemble gives bitwise the per-realisation
    # pic_step runs on the same context
    Ns = [3000, 7000, 20000, 5000, 12000]
    Ngs = [128, 256, 512, 1024, 128]
    kap = [20.0, 50.0, 200.0, 30.0, 100.0]
    us, vs = loads(Ns)
    u = to_dev_u(np.concatenate(us))
    v = to_dev(np.concatenate(vs))
    c = kp.Context(0) if cut == "tuned" else ctx
    try:
        if cut == "tuned":
            c.set_autotune(True)
        else:
            c.set_truncation(cut)
        ens = kp.Ensemble(c, Ns, Ngs, kap, L, 0.1, u, v)
        steps = 10
        en = torch.zeros(len(Ns) * steps, dtype=torch.float64, device=DEV)
        ens.run(steps, en, use_graph=True)
        c.sync()
        if cut == "tuned":
            cuts = [e for e in c.autotune_table() if e["kind"] == "cut_log2"]
            assert len(cuts) == len(set(zip(Ngs, kap)))  # one choice per key, shared by the lanes
            assert all(e["value"] in (24.0, 20.0, 18.0) for e in cuts)
        en = en.cpu().numpy().reshape(len(Ns), steps)
        off = np.concatenate([[0], np.cumsum(Ns)])
        for r in range(len(Ns)):
            st = kp.PicState(to_dev_u(us[r]), to_dev(vs[r]), L, Ngs[r], 0.1, kappa_uniform=kap[r], max_steps=steps)
            c.pic_step(st, steps)
            c.sync()
            np.testing.assert_array_equal(en[r], st.energy.cpu().numpy())
            assert torch.equal(u[off[r]:off[r + 1]], st.u) and torch.equal(v[off[r]:off[r + 1]], st.v)
        ens.close()
    finally:
        if cut == "tuned":
            c.close()
        else:
            c.set_truncation(0.0)


def test_graph_replay_equals_plain_launches_and_resume(ctx, kp):
    Ns = [4000, 9000, 2500]
    Ngs = [256, 512, 128]
    kap = [40.0, 40.0, 40.0]
    us, vs = loads(Ns, 10)
    out = []
    for use_graph, split in ((True, False), (False, False), (True, True)):
        u = to_dev_u(np.concatenate(us))
        v = to_dev(np.concatenate(vs))
        ens = kp.Ensemble(ctx, Ns, Ngs, kap, L, 0.1, u, v)
        en = torch.zeros(3 * 6, dtype=torch.float64, device=DEV)
        if split:  # two runs of three steps continue the same trajectory
            a = torch.zeros(3 * 3, dtype=torch.float64, device=DEV)
            b = torch.zeros(3 * 3, dtype=torch.float64, device=DEV)
            ens.run(3, a, use_graph=use_graph)
            ens.run(3, b, use_graph=use_graph)
            en = torch.cat([a.view(3, 3), b.view(3, 3)], dim=1).reshape(-1)
        else:
            ens.run(6, en, use_graph=use_graph)
        ctx.sync()
        out.append((u.clone(), v.clone(), en.clone()))
        ens.close()
    for k in (1, 2):
        for x, y in zip(out[0], out[k]):
            assert torch.equal(x, y)


def test_many_realisations_over_few_lanes(ctx, kp):
    R = 40
    Ns = [2048 + 97 * r for r in range(R)]
    Ngs = [(64, 100, 256)[r % 3] for r in range(R)]
    kap = [10.0 + r for r in range(R)]
    us, vs = loads(Ns, 30)
    u = to_dev_u(np.concatenate(us))
    v = to_dev(np.concatenate(vs))
    ens = kp.Ensemble(ctx, Ns, Ngs, kap, L, 0.1, u, v)
    en = torch.zeros(R * 4, dtype=torch.float64, device=DEV)
    ens.run(4, en, use_graph=True)
    ctx.sync()
    en = en.cpu().numpy().reshape(R, 4)
    off = np.concatenate([[0], np.cumsum(Ns)])
    for r in (0, 17, 39):
        st = kp.PicState(to_dev_u(us[r]), to_dev(vs[r]), L, Ngs[r], 0.1, kappa_uniform=kap[r], max_steps=4)
        ctx.pic_step(st, 4)
        ctx.sync()
        np.testing.assert_array_equal(en[r], st.energy.cpu().numpy())
        assert torch.equal(u[off[r]:off[r + 1]], st.u)
    # new widths: the captured step is captured again and follows them
    ens.set_widths([25.0] * R)
    ens.run(2, None, use_graph=True)
    ctx.sync()
    ens.close()


def test_ensemble_mise_against_oracle(ctx, kp, oracle):
    Ns = [2000, 6000, 16000]
    Ngs = [128, 512, 1024]
    kap = [10.0, 60.0, 300.0]
    us, vs = loads(Ns, 20)
    ens = kp.Ensemble(ctx, Ns, Ngs, kap, L, 0.1, to_dev_u(np.concatenate(us)), to_dev(np.concatenate(vs)))
    m = ens.mise(0.05, 1).cpu().numpy()
    for r in range(3):
        x = I.from_fixed(us[r], L)
        rho = oracle.deposit(x, Ngs[r], L, kappa_u=kap[r])
        truth = 1 + 0.05 * np.cos(2 * math.pi * np.arange(Ngs[r]) / Ngs[r])
        ref = np.sum((rho - truth) ** 2) * L / Ngs[r]
        assert m[r] == pytest.approx(ref, rel=1e-3)
    ens.close()


def test_ensemble_rejects_bad_arguments(ctx, kp):
    u = to_dev_u(np.zeros(100, dtype=np.uint32))
    v = to_dev(np.zeros(100, dtype=np.float32))
    with pytest.raises(kp.KdeError):
        kp.Ensemble(ctx, [100], [5000], [10.0], L, 0.1, u, v)
    with pytest.raises(kp.KdeError):
        kp.Ensemble(ctx, [100], [64], [0.0], L, 0.1, u, v)
    ens = kp.Ensemble(ctx, [50, 50], [64, 64], [10.0, 10.0], L, 0.1, u, v)
    with pytest.raises(kp.KdeError):
        ens.run(3, torch.zeros(5, dtype=torch.float64, device=DEV))
    ens.close()
