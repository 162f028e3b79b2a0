"""GPU parity of the cross-validation (Eq. cv_def) and Silverman widths against the oracle.

Tolerance for CV values: 2e-6 of max |CV|.  The pair term is a mean of FP32
kernel values (per-term rounding ~1e-7, independent across pairs) accumulated
in FP64; the integral term is an exact trapezoid sum whose nodes are FP32
deposits (~1e-6 relative), so 2e-6 bounds both.  The selected width must be
the oracle's unless the oracle's two best values are closer than ten times
that tolerance (then the choice is reported, not failed, and both must be
among the oracle's near-best).
"""
import math

import numpy as np
import pytest
import torch

import kde_inputs as I
from conftest import to_dev, to_dev_u

pytestmark = pytest.mark.gpu

TOL = 2e-6


def check_curve(cv, am, ref, tol=TOL, label=""):
    """CV curve within tol of max|CV|; the selected width identical to the oracle's,
    unless the oracle's two best values are a near-tie (gap <= 10 tol max|CV|).  Prints
    which branch decided (run pytest with -s to see it) and returns it."""
    scale = np.max(np.abs(ref))
    err = np.max(np.abs(cv - ref)) / scale
    assert err <= tol, err
    order = np.argsort(ref)
    gap = (ref[order[1]] - ref[order[0]]) / scale
    if gap > 10 * tol:
        branch = "identical"
        assert am == int(order[0])
    else:
        branch = "near-tie"
        assert ref[am] - ref[order[0]] <= 10 * tol * scale
    print("kappa* check %s: %s (GPU argmin %d, oracle argmin %d, oracle gap %.3e of max|CV|, "
          "GPU CV error %.3e of max|CV|)" % (label, branch, am, int(order[0]), gap, err))
    return branch


@pytest.mark.parametrize("N", [2, 3, 255, 256, 257, 3000])
def test_cv_uniform_small(ctx, oracle, N):
    L = 2 * math.pi
    u = I.cv_sweep_load(N, N)
    x = I.from_fixed(u, L)
    cand = I.log_candidates(1.0, 1e4, 16)
    cv, am, loo = ctx.cv(to_dev_u(u), L, cand, want_loo=True, pairs=True)
    if N <= 300:
        ref = np.array([oracle.cv_dense(x, L, kappa_u=c)[0] for c in cand])
        _, _, _, loo_ref = oracle.cv_dense(x, L, kappa_u=cand[am], want_loo=True)
    else:
        ref = np.array([oracle.cv_fourier(x, L, c)[0] for c in cand])
        _, _, _, loo_ref = oracle.cv_fourier(x, L, cand[am], want_loo=True)
    check_curve(cv, am, ref)
    np.testing.assert_allclose(loo.cpu().numpy(), loo_ref, rtol=1e-5, atol=1e-7 * np.max(loo_ref))


def test_cv_uniform_other_domain(ctx, oracle):
    # x units: CV scales with 2 pi / L
    L = 4 * math.pi
    u, _ = I.landau_load(4, 2000, L)
    x = I.from_fixed(u, L)
    cand = np.array([3.0, 30.0, 300.0, 3000.0])
    cv, am, _ = ctx.cv(to_dev_u(u), L, cand, pairs=True)
    ref = np.array([oracle.cv_fourier(x, L, c)[0] for c in cand])
    check_curve(cv, am, ref)


def test_cv_unsorted_candidates_and_ties(ctx, oracle):
    L = 2 * math.pi
    u = I.cv_sweep_load(5, 1000)
    x = I.from_fixed(u, L)
    cand = np.array([500.0, 2.0, 50.0, 50.0, 5000.0])
    cv, am, _ = ctx.cv(to_dev_u(u), L, cand, pairs=True)
    ref = np.array([oracle.cv_fourier(x, L, c)[0] for c in cand])
    check_curve(cv, am, ref)
    assert cv[2] == cv[3]
    if am in (2, 3):
        assert am == 2  # smallest index on an exact tie


def test_cv_scale_mode(ctx, oracle):
    L = 4 * math.pi
    N = 1500
    u, _ = I.landau_load(6, N, L)
    x = I.from_fixed(u, L)
    kr = I.log_uniform(6, I.STREAM_KAPPA, N, 5.0, 5e3).astype(np.float32)
    scales = 10.0 ** ((np.arange(16) - 8) / 8.0)
    cv, am, loo = ctx.cv(to_dev_u(u), L, scales, kappa_rel=to_dev(kr), want_loo=True)
    ref = np.array([oracle.cv_dense(x, L, kappa=s * kr.astype(np.float64))[0] for s in scales])
    check_curve(cv, am, ref)
    _, _, _, loo_ref = oracle.cv_dense(x, L, kappa=scales[am] * kr.astype(np.float64), want_loo=True)
    np.testing.assert_allclose(loo.cpu().numpy(), loo_ref, rtol=1e-5, atol=1e-7 * np.max(loo_ref))


def test_cv_duplicate_points(ctx, oracle):
    L = 1.0
    u = np.repeat(np.array([10, 2 ** 31, 3 * 2 ** 30], dtype=np.uint32), 100)
    x = I.from_fixed(u, L)
    cand = np.array([1.0, 10.0, 100.0])
    cv, am, _ = ctx.cv(to_dev_u(u), L, cand, pairs=True)
    ref = np.array([oracle.cv_fourier(x, L, c)[0] for c in cand])
    check_curve(cv, am, ref)


def test_cv_rejects_bad_arguments(ctx, kp):
    u = to_dev_u(np.arange(10, dtype=np.uint32))
    with pytest.raises(kp.KdeError):
        ctx.cv(u[:1], 1.0, [1.0])
    with pytest.raises(kp.KdeError):
        ctx.cv(u, 1.0, [0.0])
    with pytest.raises(kp.KdeError):
        ctx.cv(u, 1.0, np.ones(300))


def test_cv_deterministic(ctx):
    L = 2 * math.pi
    u = to_dev_u(I.cv_sweep_load(3, 50_000))
    cand = I.log_candidates(1.0, 1e4, 8)
    a, _, la = ctx.cv(u, L, cand, want_loo=True, pairs=True)
    b, _, lb = ctx.cv(u, L, cand, want_loo=True, pairs=True)
    assert np.array_equal(a, b) and torch.equal(la, lb)


def test_cv_sweep_full_size(ctx, oracle):
    # the CV-sweep workload: N = 2^18 mixture positions, 64 candidates in [1, 1e4]
    L = 2 * math.pi
    u = I.cv_sweep_load(0, 1 << 18)
    x = I.from_fixed(u, L)
    cand = I.log_candidates(1.0, 1e4, 64)
    cv, am, loo = ctx.cv(to_dev_u(u), L, cand, want_loo=True, pairs=True)
    ref = np.array([oracle.cv_fourier(x, L, c)[0] for c in cand])
    check_curve(cv, am, ref, label="CV sweep N=2^18 x 64")
    _, _, _, loo_ref = oracle.cv_fourier(x, L, cand[am], want_loo=True)
    idx = np.arange(0, 1 << 18, 61)
    np.testing.assert_allclose(loo.cpu().numpy()[idx], loo_ref[idx], rtol=1e-5, atol=1e-7 * np.max(loo_ref))


def test_adapt_widths(ctx, oracle):
    L = 2 * math.pi
    N = 20_000
    u = I.cv_sweep_load(2, N)
    x = I.from_fixed(u, L)
    _, _, _, loo = oracle.cv_fourier(x, L, 300.0, want_loo=True)
    loo32 = loo.astype(np.float32)
    k = ctx.adapt_widths(to_dev(loo32), L, 300.0, 0.5, 10.0, 1e4).cpu().numpy()
    ref = oracle.adapt_widths(loo32.astype(np.float64), L, 300.0, 0.5, 10.0, 1e4)
    np.testing.assert_allclose(k, ref, rtol=2e-6)


# ---------------------------------------------------------------------------
# exact Fourier form of the CV (uniform widths)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N", [2000, 3001])
def test_cv_spectral_against_dense(ctx, oracle, N):
    L = 4 * math.pi
    u, _ = I.landau_load(N, N, L, 0.05, 1.0)
    x = I.from_fixed(u, L)
    cand = I.log_candidates(1.0, 1e4, 16)
    cv, am, loo = ctx.cv(to_dev_u(u), L, cand, want_loo=True, spectral=True)
    ref = np.array([oracle.cv_dense(x, L, kappa_u=c)[0] for c in cand])
    # an exact identity combined in FP64; the phases are FP32 sincospi of exact
    # 32-bit turn fractions (~1e-7 per term), so 1e-8 of max |CV| bounds the error
    check_curve(cv, am, ref, tol=1e-8)
    _, _, _, loo_ref = oracle.cv_dense(x, L, kappa_u=cand[am], want_loo=True)
    np.testing.assert_allclose(loo.cpu().numpy(), loo_ref, rtol=1e-5, atol=1e-7 * np.max(loo_ref))


def test_cv_spectral_matches_pairs_and_sweep_size(ctx, oracle):
    L = 2 * math.pi
    u = I.cv_sweep_load(0, 1 << 18)
    x = I.from_fixed(u, L)
    cand = I.log_candidates(1.0, 1e4, 64)
    ud = to_dev_u(u)
    cs, ams, ls = ctx.cv(ud, L, cand, want_loo=True, spectral=True)
    cp, amp, lp = ctx.cv(ud, L, cand, want_loo=True, pairs=True)
    sel = np.arange(0, 64, 7)
    ref = np.array([oracle.cv_fourier(x, L, cand[c])[0] for c in sel])
    assert np.max(np.abs(cs[sel] - ref)) <= 1e-8 * np.max(np.abs(ref))
    assert np.max(np.abs(cs - cp)) <= TOL * np.max(np.abs(cs))
    assert ams == amp or abs(cs[amp] - cs[ams]) <= 10 * TOL * np.max(np.abs(cs))
    idx = np.arange(0, 1 << 18, 97)
    np.testing.assert_allclose(ls.cpu().numpy()[idx], lp.cpu().numpy()[idx], rtol=2e-5)


def test_cv_spectral_ratio_table_reuse(ctx, kp):
    # the Bessel-ratio table of a candidate list is kept between calls and reused when
    # the same list comes back; a different list (even one of the same length) must be
    # worked out again: results equal those of a fresh context, bit for bit
    L = 2 * math.pi
    u = to_dev_u(I.cv_sweep_load(4, 20000))
    a = I.log_candidates(1.0, 1e4, 16)
    b = I.log_candidates(2.0, 5e3, 16)
    runs = []
    for cands in (a, a, b, a, b[::-1]):
        cv, am, loo = ctx.cv(u, L, cands, want_loo=True, spectral=True)
        runs.append((cv, am, loo.cpu().numpy()))
    fresh = kp.Context(0)
    try:
        for cands, (cv, am, loo) in zip((a, a, b, a, b[::-1]), runs):
            cv2, am2, loo2 = fresh.cv(u, L, cands, want_loo=True, spectral=True)
            fresh.close()
            fresh = kp.Context(0)
            np.testing.assert_array_equal(cv, cv2)
            assert am == am2
            np.testing.assert_array_equal(loo, loo2.cpu().numpy())
    finally:
        fresh.close()


def test_cv_spectral_rejects_scale_mode(ctx, kp):
    u = to_dev_u(np.arange(100, dtype=np.uint32) * 40000)
    with pytest.raises(kp.KdeError):
        ctx.cv(u, 1.0, [1.0, 2.0], kappa_rel=to_dev(np.ones(100)), spectral=True)


def test_bounded_wait_gives_up_and_context_recovers(kp, oracle):
    # the tile waits of the CV kernels are bounded: with a limit of zero polls every
    # wait gives up, the kernels drain their copies in flight and flag the status
    # word, kde_cv reports KDE_EDEVICE, and the same context then computes the
    # right curve again (uniform widths: the persistent kernel; scale mode: the
    # tile kernel)
    c = kp.Context(0)
    try:
        L = 2 * math.pi
        N = 3000
        u = I.cv_sweep_load(5, N)
        x = I.from_fixed(u, L)
        ud = to_dev_u(u)
        cand = I.log_candidates(1.0, 1e4, 12)
        kr = I.log_uniform(5, 0, N, 0.5, 2.0).astype(np.float32)
        scales = I.log_candidates(1.0, 1e3, 6)
        for kw in ({}, {"kappa_rel": to_dev(kr)}):
            c.set_wait_limit(0)
            with pytest.raises(kp.KdeError) as e:
                c.cv(ud, L, scales if kw else cand, pairs=not kw, **kw)
            assert e.value.code == 4 and "wait" in str(e.value)
            c.set_wait_limit(-1)
            if kw:
                cv, am, _ = c.cv(ud, L, scales, **kw)
                ref = oracle.cv_curve(x, L, scales, kappa_rel=kr.astype(np.float64))
            else:
                cv, am, _ = c.cv(ud, L, cand, pairs=True)
                ref = oracle.cv_curve(x, L, cand, fourier=True)
            check_curve(cv, am, ref)
    finally:
        c.close()


def test_cv_cost_rule_picks_an_exact_form(ctx, oracle, kp):
    # without a form flag the library takes the cheaper exact form: at N = 2^15 with
    # candidates up to 1e4 the Fourier form (bitwise its result), at N = 40 the pair
    # sums (bitwise theirs); both agree with the oracle; the two flags together are refused
    L = 4 * math.pi
    cand = I.log_candidates(1.0, 1e4, 16)
    for N, form in ((1 << 15, "spectral"), (40, "pairs")):
        u, _ = I.landau_load(21, N, L, 0.05, 1.0)
        ud = to_dev_u(u)
        auto, am, la = ctx.cv(ud, L, cand, want_loo=True)
        forced, amf, lf = ctx.cv(ud, L, cand, want_loo=True, **{form: True})
        assert np.array_equal(auto, forced) and am == amf
        assert torch.equal(la, lf)
        ref = oracle.cv_curve(I.from_fixed(u, L), L, cand, fourier=True)
        check_curve(auto, am, ref, label="cost rule N=%d (%s)" % (N, form))
    with pytest.raises(kp.KdeError):
        ctx.cv(ud, L, cand, spectral=True, pairs=True)
