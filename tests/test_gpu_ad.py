"""GPU parity of the Anderson-Darling test and of the Sec. II.D width-update schedule.

* kde_ad_test against the oracle's A^2 (its own sort and the textbook sum) on the same
  position codes, across sizes that span several blocks and a ragged tail, uniform,
  perturbed, clustered, tied and extreme codes, and the full 2^20 Landau load; the FP32
  in-bin logarithms bound the error by about 2e-11 N in A^2;
* ln p through the same published expressions within that error;
* bitwise determinism and argument checks;
* pic_step with width_ad in FP64 against the oracle's PIC run driven by the same rule:
  the same optimisation steps, the same widths and ln p per step, the same energies.
"""
import math

import numpy as np
import pytest
import torch

import kde_inputs as I
from conftest import to_dev, to_dev_u

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
L = 4 * math.pi


def a2_tol(N, a2):
    return 2e-11 * N + 1e-12 * abs(a2) + 1e-12


def check(ctx, oracle, u):
    a2, lp = ctx.ad_test(to_dev_u(u))
    ref = oracle.ad_statistic(oracle.ad_cdf_of_codes(u))
    assert abs(a2 - ref) <= a2_tol(u.size, ref), (a2, ref)
    # ln p from the published expressions: both sides agree to the A^2 error (d ln p / dA^2 >~ -1.5)
    lref = oracle.ad_log_pvalue(ref, u.size)
    assert abs(lp - lref) <= 2.0 * a2_tol(u.size, ref) + 1e-9 * abs(lref), (lp, lref)
    return a2, lp


@pytest.mark.parametrize("N", [8, 9, 2047, 2048, 2049, 5000, 65537])
def test_uniform_random_sizes(ctx, oracle, N):
    u = I.to_fixed(I.random_positions(5, N, L, 0.0), L)
    check(ctx, oracle, u)


def test_perturbed_clustered_and_quiet(ctx, oracle):
    u = I.to_fixed(I.random_positions(6, 30000, L, 0.3), L)
    a2, lp = check(ctx, oracle, u)
    assert a2 > 50 and lp < -40  # clearly not uniform; ln p does not underflow
    check(ctx, oracle, I.cv_sweep_load(1, 1 << 16))  # 0.7 uniform + 0.3 von Mises(pi, 20)
    q = I.to_fixed(I.quiet_positions(4096, L, 0.0), L)
    a2, lp = check(ctx, oracle, q)
    assert a2 < 0.01 and lp > -1e-3


def test_ties_and_extreme_codes(ctx, oracle):
    rng = np.random.default_rng(3)
    u = rng.integers(0, 4, 4096).astype(np.uint32) * np.uint32(1 << 30) + np.uint32(12345)  # four tied values
    check(ctx, oracle, u)
    u = np.concatenate([np.zeros(100, np.uint32), np.full(100, 2 ** 32 - 1, np.uint32),
                        rng.integers(0, 2 ** 32, 3000, dtype=np.uint64).astype(np.uint32)])
    check(ctx, oracle, u)
    u = np.full(5000, 777, dtype=np.uint32)  # every particle at one code
    check(ctx, oracle, u)


def test_full_size_landau(ctx, oracle):
    u, _ = I.landau_load(0, 1 << 20, L, 0.05, 1.0)
    a2, lp = check(ctx, oracle, u)
    assert a2 > 20


def test_deterministic_and_input_untouched(ctx):
    u, _ = I.landau_load(1, 300001, L, 0.05, 1.0)
    du = to_dev_u(u)
    a = ctx.ad_test(du)
    b = ctx.ad_test(du)
    assert a == b
    np.testing.assert_array_equal(du.cpu().numpy().view(np.uint32), u)


def test_rejects_small_samples(ctx, kp):
    with pytest.raises(kp.KdeError):
        ctx.ad_test(to_dev_u(np.arange(7, dtype=np.uint32)))


def run_pair(ctx, kp, oracle, u, v, Ng, dt, steps, k0, cand, spectral=False):
    st = kp.PicState(to_dev_u(u), to_dev(v, torch.float64), L, Ng, dt, kappa_uniform=k0, cand=cand,
                     max_steps=steps, width_ad=True, cv_spectral=spectral)
    ctx.pic_step(st, steps)
    ctx.sync()
    r = oracle.pic_run_ad(I.from_fixed(u, L), v, L, Ng, dt, steps, k0, cand)
    return st, r


def test_schedule_matches_oracle_fp64(ctx, kp, oracle):
    N, Ng, dt, steps = 4096, 64, 0.1, 40
    u, v = I.landau_load(8, N, L, 0.3, 1.0)
    cand = I.log_candidates(1.0, 1e3, 16)
    st, r = run_pair(ctx, kp, oracle, u, v, Ng, dt, steps, 20.0, cand, spectral=True)
    lp = st.ad_log_p.cpu().numpy()[:steps]
    # decisions are compared only where they are not near-ties of the halving rule
    np.testing.assert_allclose(lp, r["log_pvalue"], rtol=1e-9, atol=1e-6)
    assert st.c.n_opt == int(r["optimised"].sum()) and st.c.n_opt >= 1
    np.testing.assert_allclose(st.kappa_star.cpu().numpy()[:steps], r["kappa"], rtol=1e-10)
    assert st.c.kappa_uniform == pytest.approx(r["kappa_u"], rel=1e-12)
    assert st.c.h_target == pytest.approx(r["h_target"], rel=1e-12)
    assert st.c.ad_log_pth == pytest.approx(r["lp_th"], rel=1e-9, abs=1e-6)
    W = st.energy.cpu().numpy()[:steps]
    np.testing.assert_allclose(W, r["energy"], rtol=0, atol=1e-7 * r["energy"].max())


def test_schedule_pairs_cv_and_resume(ctx, kp, oracle):
    # pair-sum CV selects the same targets; two calls of n steps equal one call of 2n
    N, Ng, dt = 4096, 64, 0.1
    u, v = I.landau_load(9, N, L, 0.3, 1.0)
    cand = I.log_candidates(1.0, 1e3, 16)
    a, r = run_pair(ctx, kp, oracle, u, v, Ng, dt, 20, 20.0, cand, spectral=False)
    np.testing.assert_allclose(a.kappa_star.cpu().numpy()[:20], r["kappa"], rtol=1e-10)
    b = kp.PicState(to_dev_u(u), to_dev(v, torch.float64), L, Ng, dt, kappa_uniform=20.0, cand=cand,
                    max_steps=20, width_ad=True)
    ctx.pic_step(b, 10)
    ctx.pic_step(b, 10)
    ctx.sync()
    assert torch.equal(a.u, b.u) and torch.equal(a.v, b.v)
    assert torch.equal(a.ad_log_p, b.ad_log_p) and a.c.n_opt == b.c.n_opt


def test_schedule_fp32_runs_and_rejects_particle_widths(ctx, kp):
    N, Ng, dt = 1 << 16, 256, 0.1
    u, v = I.landau_load(10, N, L, 0.05, 1.0)
    cand = I.log_candidates(1.0, 1e4, 32)
    st = kp.PicState(to_dev_u(u), to_dev(v), L, Ng, dt, kappa_uniform=50.0, cand=cand, max_steps=30,
                     width_ad=True, cv_spectral=True)
    ctx.pic_step(st, 30)
    ctx.sync()
    lp = st.ad_log_p.cpu().numpy()[:30]
    assert np.all(np.isfinite(lp)) and st.c.n_opt >= 1
    bad = kp.PicState(to_dev_u(u), to_dev(v), L, Ng, dt, kappa=to_dev(np.full(N, 50.0)), cand=cand,
                      max_steps=2, width_ad=True)
    with pytest.raises(kp.KdeError):
        ctx.pic_step(bad, 1)
