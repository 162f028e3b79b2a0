"""GPU parity of deposit, Poisson and gather (through the C ABI) against the FP64 oracle.

Tolerances: FP32 results within 1e-5 relative L2 of the oracle (density and
field, as required of the FP32 path); FP64 results within 1e-10 relative L2
(FP64 arithmetic, truncation below 2^-64 of each kernel's peak, int64 grid
accumulation with a quantum below 1e-15 of the mean density).
"""
import math

import numpy as np
import pytest
import torch

import kde_inputs as I
from conftest import rel_l2, to_dev, to_dev_u

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-10


def landau(seed, N, L=4 * math.pi):
    u, v = I.landau_load(seed, N, L, 0.05, 1.0)
    return u, I.from_fixed(u, L), v


@pytest.mark.parametrize("N", [1, 31, 1000, 70001])
@pytest.mark.parametrize("Ng,kappa", [(64, 0.5), (64, 30.0), (100, 300.0), (256, 3000.0), (4096, 1e4), (33, 8.0)])
def test_deposit_uniform_fp32(ctx, oracle, N, Ng, kappa):
    L = 4 * math.pi
    u, x, _ = landau(N + Ng, N, L)
    rho = ctx.deposit(to_dev_u(u), Ng, L, kappa_uniform=kappa).cpu().numpy()
    ref = oracle.deposit(x, Ng, L, kappa_u=kappa)
    assert rel_l2(rho, ref) <= TOL32


@pytest.mark.parametrize("Ng", [64, 100, 256])
def test_deposit_per_particle_and_weights(ctx, oracle, Ng):
    L = 4 * math.pi
    N = 5000
    u, x, _ = landau(3, N, L)
    k = I.log_uniform(3, I.STREAM_KAPPA, N, 5.0, 5e3)
    w = 0.5 + I.uniforms(3, 9, N)
    rho = ctx.deposit(to_dev_u(u), Ng, L, kappa=to_dev(k), weight=to_dev(w)).cpu().numpy()
    ref = oracle.deposit(x, Ng, L, kappa=k.astype(np.float32), w=w.astype(np.float32))
    assert rel_l2(rho, ref) <= TOL32
    rho2 = ctx.deposit(to_dev_u(u), Ng, L, kappa=to_dev(k)).cpu().numpy()
    assert rel_l2(rho2, oracle.deposit(x, Ng, L, kappa=k.astype(np.float32))) <= TOL32


@pytest.mark.parametrize("Ng,kappa", [(64, 3.0), (64, 200.0), (100, 1000.0)])
def test_deposit_fp64(ctx, oracle, Ng, kappa):
    L = 4 * math.pi
    N = 4096
    u, x, _ = landau(5, N, L)
    rho = ctx.deposit(to_dev_u(u), Ng, L, kappa_uniform=kappa, dtype=torch.float64).cpu().numpy()
    assert rel_l2(rho, oracle.deposit(x, Ng, L, kappa_u=kappa)) <= TOL64
    k = I.log_uniform(5, I.STREAM_KAPPA, N, 5.0, 500.0)
    rho = ctx.deposit(to_dev_u(u), Ng, L, kappa=to_dev(k, torch.float64)).cpu().numpy()
    assert rel_l2(rho, oracle.deposit(x, Ng, L, kappa=k)) <= TOL64


def test_deposit_edge_cases(ctx, oracle):
    L = 1.0
    # empty input gives zeros
    rho = ctx.deposit(to_dev_u(np.zeros(0, np.uint32)), 16, L, kappa_uniform=5.0).cpu().numpy()
    assert np.all(rho == 0)
    # one-node and two-node grids
    u, x, _ = landau(1, 300, L)
    for Ng in (1, 2):
        rho = ctx.deposit(to_dev_u(u), Ng, L, kappa_uniform=50.0).cpu().numpy()
        assert rel_l2(rho, oracle.deposit(x, Ng, L, kappa_u=50.0)) <= TOL32
    # all particles in one cell and on the wrap-around point
    uu = np.full(2000, 0xFFFFFFF0, np.uint32)
    uu[::2] = 5
    rho = ctx.deposit(to_dev_u(uu), 128, L, kappa_uniform=2000.0).cpu().numpy()
    assert rel_l2(rho, oracle.deposit(I.from_fixed(uu, L), 128, L, kappa_u=2000.0)) <= TOL32


def test_deposit_is_deterministic(ctx):
    L = 4 * math.pi
    u, _, _ = landau(8, 100_000, L)
    ud = to_dev_u(u)
    a = ctx.deposit(ud, 256, L, kappa_uniform=400.0)
    b = ctx.deposit(ud, 256, L, kappa_uniform=400.0)
    assert torch.equal(a, b)


def test_deposit_rejects_bad_arguments(ctx, kp):
    u = to_dev_u(np.arange(10, dtype=np.uint32))
    with pytest.raises(kp.KdeError):
        ctx.deposit(u, 5000, 1.0, kappa_uniform=5.0)
    with pytest.raises(kp.KdeError):
        ctx.deposit(u, 16, 1.0, kappa_uniform=-1.0)
    with pytest.raises(kp.KdeError):
        ctx.deposit(u, 16, -1.0, kappa_uniform=1.0)


def test_device_status_reports_bad_width(ctx, kp):
    u = to_dev_u(np.arange(10, dtype=np.uint32) * 1000)
    k = to_dev(np.array([5.0] * 9 + [-3.0]))
    ctx.deposit(u, 16, 1.0, kappa=k)
    with pytest.raises(kp.KdeError):
        ctx.sync()
    ctx.sync()  # the status word was cleared


@pytest.mark.parametrize("Ng", [1, 2, 3, 64, 100, 256, 1000, 4096])
@pytest.mark.parametrize("fd", [False, True])
def test_poisson(ctx, oracle, Ng, fd):
    L = 4 * math.pi
    r = 1.0 + 0.05 * np.cos(2 * math.pi * np.arange(Ng) / Ng) + 0.01 * (I.uniforms(Ng, 4, Ng) - 0.5)
    E = ctx.poisson(to_dev(r), L, fd=fd).cpu().numpy()
    ref = oracle.poisson(1.0 - r, L, fd=fd)
    assert np.linalg.norm(E - ref) <= TOL32 * max(np.linalg.norm(ref), 1e-30) + 1e-12
    E64 = ctx.poisson(to_dev(r, torch.float64), L, fd=fd).cpu().numpy()
    assert np.linalg.norm(E64 - ref) <= TOL64 * max(np.linalg.norm(ref), 1e-30) + 1e-14


def test_poisson_energy(ctx, oracle):
    L = 4 * math.pi
    r = 1.0 + 0.05 * np.cos(2 * math.pi * np.arange(256) / 256)
    en = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    E = ctx.poisson(to_dev(r, torch.float64), L, energy=en)
    ref = oracle.field_energy(oracle.poisson(1.0 - r, L), L)
    assert en.item() == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("N", [1, 37, 5000])
@pytest.mark.parametrize("Ng,kappa", [(64, 1.0), (64, 50.0), (100, 500.0), (256, 4000.0), (4096, 1e4)])
def test_gather_uniform(ctx, oracle, N, Ng, kappa):
    L = 4 * math.pi
    u, x, _ = landau(N * 7 + Ng, N, L)
    f = np.sin(2 * math.pi * np.arange(Ng) / Ng) + 0.3 * np.cos(6 * math.pi * np.arange(Ng) / Ng)
    out = ctx.gather(to_dev_u(u), to_dev(f), L, kappa_uniform=kappa).cpu().numpy()
    ref = oracle.gather(x, f.astype(np.float32), L, kappa_u=kappa)
    assert rel_l2(out, ref) <= TOL32


def test_gather_per_particle_and_fp64(ctx, oracle):
    L = 4 * math.pi
    N, Ng = 4000, 128
    u, x, _ = landau(11, N, L)
    k = I.log_uniform(11, I.STREAM_KAPPA, N, 5.0, 5e3)
    f = np.cos(2 * math.pi * np.arange(Ng) / Ng)
    out = ctx.gather(to_dev_u(u), to_dev(f), L, kappa=to_dev(k)).cpu().numpy()
    assert rel_l2(out, oracle.gather(x, f, L, kappa=k.astype(np.float32))) <= TOL32
    out64 = ctx.gather(to_dev_u(u), to_dev(f, torch.float64), L, kappa=to_dev(k, torch.float64)).cpu().numpy()
    assert rel_l2(out64, oracle.gather(x, f, L, kappa=k)) <= TOL64


@pytest.mark.parametrize("kappa", [0.3, 12.0, 32.0, 32.5, 90.0])
def test_kernel_value_forms(ctx, oracle, kappa):
    # widths up to 32 take the cosine form of the FP32 kernel value (three multiply-adds
    # a pair, an exponent that loses about K 2^-24 near the peak), wider ones the
    # half-angle form; both stay within a few 1e-7 of the oracle in L2 on this load
    L = 4 * math.pi
    N, Ng = 20000, 256
    u, x, _ = landau(17, N, L)
    rho = ctx.deposit(to_dev_u(u), Ng, L, kappa_uniform=kappa).cpu().numpy()
    assert rel_l2(rho, oracle.deposit(x, Ng, L, kappa_u=kappa)) <= 2e-6
    f = np.sin(2 * math.pi * np.arange(Ng) / Ng) + 0.5
    out = ctx.gather(to_dev_u(u), to_dev(f), L, kappa_uniform=kappa).cpu().numpy()
    assert rel_l2(out, oracle.gather(x, f.astype(np.float32), L, kappa_u=kappa)) <= 2e-6


def test_kernel_value_forms_mixed_chunks(ctx, oracle):
    # narrow kernels on one half of the box, wide ones on the other: chunks and blocks
    # of either form and the ones that straddle the change
    L = 4 * math.pi
    N, Ng = 30000, 128
    u, x, _ = landau(23, N, L)
    k = (np.where(x < L / 2, 10.0, 80.0) * (0.9 + 0.2 * I.uniforms(23, 9, N))).astype(np.float32)
    rho = ctx.deposit(to_dev_u(u), Ng, L, kappa=to_dev(k)).cpu().numpy()
    assert rel_l2(rho, oracle.deposit(x, Ng, L, kappa=k.astype(np.float64))) <= 2e-6
    f = np.cos(2 * math.pi * np.arange(Ng) / Ng)
    out = ctx.gather(to_dev_u(u), to_dev(f), L, kappa=to_dev(k)).cpu().numpy()
    assert rel_l2(out, oracle.gather(x, f, L, kappa=k.astype(np.float64))) <= 2e-6


def test_full_size_landau_deposit_gather_narrow(ctx, oracle):
    # the Landau workload with the widths that Silverman's rule gives it (kappa ~ 8-30),
    # which run in the cosine form
    L = 4 * math.pi
    N, Ng = 1 << 20, 256
    u, x, _ = landau(4, N, L)
    k = I.log_uniform(4, I.STREAM_KAPPA, N, 8.0, 30.0).astype(np.float32)
    ud = to_dev_u(u)
    rho = ctx.deposit(ud, Ng, L, kappa=to_dev(k)).cpu().numpy()
    ref = oracle.deposit(x, Ng, L, kappa=k.astype(np.float64))
    assert rel_l2(rho, ref) <= TOL32
    f = oracle.poisson(1.0 - ref, L)
    out = ctx.gather(ud, to_dev(f), L, kappa=to_dev(k)).cpu().numpy()
    idx = np.linspace(0, N - 1, 4096).astype(np.int64)
    refg = oracle.gather(x[idx], f.astype(np.float32), L, kappa=k[idx].astype(np.float64))
    assert rel_l2(out[idx], refg) <= TOL32


def test_full_size_landau_deposit_gather(ctx, oracle):
    # the Landau workload: N = 2^20, Ng = 256, particle-wise widths; every node of the
    # deposit and a sample of gathered particles against the oracle
    L = 4 * math.pi
    N, Ng = 1 << 20, 256
    u, x, _ = landau(0, N, L)
    k = I.log_uniform(0, I.STREAM_KAPPA, N, 200.0, 2000.0).astype(np.float32)
    ud = to_dev_u(u)
    rho = ctx.deposit(ud, Ng, L, kappa=to_dev(k)).cpu().numpy()
    ref = oracle.deposit(x, Ng, L, kappa=k.astype(np.float64))
    assert rel_l2(rho, ref) <= TOL32
    f = oracle.poisson(1.0 - ref, L)
    out = ctx.gather(ud, to_dev(f), L, kappa=to_dev(k)).cpu().numpy()
    idx = np.linspace(0, N - 1, 4096).astype(np.int64)
    refg = oracle.gather(x[idx], f.astype(np.float32), L, kappa=k[idx].astype(np.float64))
    assert rel_l2(out[idx], refg) <= TOL32


def test_max_size_sampled(ctx, oracle):
    # the largest request size: N = 2^22 particles on 4096 nodes; sampled nodes
    L = 4 * math.pi
    N, Ng = 1 << 22, 4096
    u, x, _ = landau(2, N, L)
    k = I.log_uniform(2, I.STREAM_KAPPA, N, 5.0, 5e3).astype(np.float32)
    rho = ctx.deposit(to_dev_u(u), Ng, L, kappa=to_dev(k)).cpu().numpy()
    g = np.arange(0, Ng, 97)
    ref = oracle.kde_at(x, g * L / Ng, L, kappa=k.astype(np.float64))
    assert rel_l2(rho[g], ref) <= TOL32


def test_gather_autotune_keeps_results(ctx, kp):
    # the gather's tile shapes give bitwise-identical results; the tuner times them on
    # the first call of each key and keeps the fastest for later calls
    L = 4 * math.pi
    N, Ng = 30001, 256
    u, _, _ = landau(31, N, L)
    f = np.sin(2 * math.pi * np.arange(Ng) / Ng) + 0.2
    k = I.log_uniform(31, I.STREAM_KAPPA, N, 5.0, 500.0).astype(np.float32)
    ud, fd = to_dev_u(u), to_dev(f)
    refs = [ctx.gather(ud, fd, L, kappa_uniform=ku).cpu().numpy() for ku in (4.0, 300.0)]
    refs.append(ctx.gather(ud, fd, L, kappa=to_dev(k)).cpu().numpy())
    c2 = kp.Context(0)
    try:
        c2.set_autotune(True)
        for rep in range(2):
            outs = [c2.gather(ud, fd, L, kappa_uniform=ku).cpu().numpy() for ku in (4.0, 300.0)]
            outs.append(c2.gather(ud, fd, L, kappa=to_dev(k)).cpu().numpy())
            for a, b in zip(outs, refs):
                np.testing.assert_array_equal(a, b)
        assert c2.autotune_entries() == 3
        # pic_step with the tile-shape tuner on gives the same run bit for bit (the
        # truncation cut held at the default, which the other tuner could change)
        c2.set_truncation(24.0)
        uu, vv = I.landau_load(32, 20000, L, 0.05, 1.0)
        kk = I.log_uniform(32, I.STREAM_KAPPA, 20000, 5.0, 50.0).astype(np.float32)
        runs = []
        for c in (ctx, c2):
            st = kp.PicState(to_dev_u(uu), to_dev(vv.astype(np.float32)), L, 128, 0.1, kappa=to_dev(kk), max_steps=4)
            c.pic_step(st, 4)
            c.sync()
            runs.append((st.energy.cpu().numpy(), st.u.cpu().numpy(), st.v.cpu().numpy()))
        for a, b in zip(*runs):
            np.testing.assert_array_equal(a, b)
        assert c2.autotune_entries() == 4
    finally:
        c2.close()


@pytest.mark.parametrize("cut", [24.0, 20.0, 18.0, 16.0])
def test_truncation_cut_within_tolerance(ctx, oracle, cut):
    # every cut kde_set_truncation accepts keeps the FP32 deposit and gather within the
    # 1e-5 tolerance of the untruncated oracle; kappa = 7.3 sits near the width whose
    # kernel mass beyond the cut is largest, kappa = 300 has a window well inside the grid
    L, N = 4 * math.pi, 30001
    u, x, _ = landau(77, N, L)
    k = I.log_uniform(77, I.STREAM_KAPPA, N, 5.0, 5e3)
    ud = to_dev_u(u)
    base = {}
    try:
        for c in (24.0, cut):
            ctx.set_truncation(c)
            for Ng, kw, okw in ((256, dict(kappa_uniform=7.3), dict(kappa_u=7.3)),
                                (512, dict(kappa_uniform=300.0), dict(kappa_u=300.0)),
                                (512, dict(kappa=to_dev(k)), dict(kappa=k.astype(np.float32)))):
                rho = ctx.deposit(ud, Ng, L, **kw).cpu().numpy()
                assert rel_l2(rho, oracle.deposit(x, Ng, L, **okw)) <= TOL32
                f = np.sin(2 * math.pi * np.arange(Ng) / Ng) + 0.3
                out = ctx.gather(ud, to_dev(f), L, **kw).cpu().numpy()
                assert rel_l2(out, oracle.gather(x, f.astype(np.float32), L, **okw)) <= TOL32
                key = (Ng, str(sorted(okw)), float(okw.get("kappa_u", 0)))
                if c == 24.0:
                    base[key] = (rho, out)
                elif key[2] == 300.0:
                    # the cut reaches the kernels: a narrower window changes the sums
                    assert not np.array_equal(rho, base[key][0])
                    assert not np.array_equal(out, base[key][1])
    finally:
        ctx.set_truncation(0.0)


def test_truncation_setting_is_checked(ctx, kp):
    for bad in (15.0, 41.0, -1.0, float("nan")):
        with pytest.raises(kp.KdeError):
            ctx.set_truncation(bad)
    ctx.set_truncation(0.0)
