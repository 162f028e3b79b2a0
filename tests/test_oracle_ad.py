"""Pins of the oracle's Anderson-Darling test and width-update rule (Sec. II.D) against facts
that do not come from the oracle: the integral definition of A^2, the limiting distribution's
mean and classical percentage points, Monte Carlo of the finite-n distribution, a scripted
sequence of the update rule, and special cases of the PIC run."""
import math

import numpy as np
import pytest
from scipy import integrate

import kde_inputs as I
import oracle as O


def ad_by_integral(F):
    """A^2 = n int_0^1 (F_n(t) - t)^2 / (t (1 - t)) dt, the empirical CDF F_n being a step
    function: quadrature piece by piece between the ordered values."""
    F = np.sort(np.asarray(F, dtype=np.float64))
    n = F.size
    edges = np.concatenate([[0.0], F, [1.0]])
    total = 0.0
    for j in range(n + 1):
        c = j / n
        a, b = edges[j], edges[j + 1]
        if b > a:
            total += integrate.quad(lambda t: (c - t) ** 2 / (t * (1.0 - t)), a, b, epsabs=1e-14,
                                    epsrel=1e-13, limit=200)[0]
    return n * total


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_statistic_equals_integral_definition(n):
    rng = np.random.default_rng(100 + n)
    for _ in range(4):
        F = rng.random(n)
        assert O.ad_statistic(F) == pytest.approx(ad_by_integral(F), rel=1e-9, abs=1e-12)


def test_statistic_order_and_reflection_invariant():
    rng = np.random.default_rng(7)
    F = rng.random(50) ** 2  # skewed sample
    a = O.ad_statistic(F)
    assert O.ad_statistic(rng.permutation(F)) == pytest.approx(a, rel=1e-13)
    # reversing the axis (t -> 1 - t) leaves the uniform hypothesis and A^2 unchanged
    assert O.ad_statistic(1.0 - F) == pytest.approx(a, rel=1e-12)
    # a grossly non-uniform sample gives a large statistic
    assert a > 3.0


def test_limiting_distribution_mean_is_one():
    # E[A^2] of the limiting distribution = sum_j 1 / (j (j + 1)) = 1
    m = integrate.quad(lambda z: 1.0 - O.ad_cdf(z, 10 ** 9), 0.0, 60.0, limit=400)[0]
    assert m == pytest.approx(1.0, abs=1e-4)


@pytest.mark.parametrize("z,p", [(1.933, 0.10), (2.492, 0.05)])
def test_classical_percentage_points(z, p):
    # Anderson & Darling (1954): upper 10% and 5% points of the limiting distribution
    assert O.ad_pvalue(z, 10 ** 9) == pytest.approx(p, abs=1e-4)


@pytest.mark.parametrize("n", [5, 8, 32])
def test_finite_n_distribution_by_monte_carlo(n):
    rng = np.random.default_rng(1000 + n)
    reps = 400_000
    U = np.sort(rng.random((reps, n)), axis=1)
    i = np.arange(1, n + 1)
    A = -n - np.sum((2 * i - 1) * (np.log(U) + np.log(1.0 - U[:, ::-1])), axis=1) / n
    for z in (0.3, 0.6, 1.0, 2.0, 3.0, 4.5):
        emp = float(np.mean(A <= z))
        se = math.sqrt(max(emp * (1 - emp), 1e-6) / reps)
        assert abs(O.ad_cdf(z, n) - emp) < 5 * se + 3e-4, (n, z)


def test_pvalue_monotone_bounded_and_tail():
    zs = np.linspace(0.05, 40, 800)
    for n in (8, 4096, 1 << 20):
        lp = np.array([O.ad_log_pvalue(z, n) for z in zs])
        assert np.all(lp <= 0) and np.all(np.diff(lp) <= 0)
        assert np.all(np.diff(lp[zs > 0.5]) < 0)
        # continuous where the fitted expressions hand over to the tail (A^2 = 7)
        a, b = O.ad_log_pvalue(7.0 - 1e-9, n), O.ad_log_pvalue(7.0 + 1e-9, n)
        assert abs(a - b) < 1e-6
    # no underflow for the huge statistics of clustered samples
    assert np.isfinite(O.ad_log_pvalue(1e5, 4096)) and O.ad_log_pvalue(1e5, 4096) < -9e4


def test_tail_law_agrees_with_fitted_distribution():
    # The limiting A^2 is sum_j chi^2_1 / (j (j + 1)); its tail is dominated by the j = 1
    # term: P(A^2 > z) ~ sqrt(3) e^{-z} / sqrt(pi z) (the sqrt(3) is the product over the
    # other weights of (1 - w_j / w_1)^{-1/2}).  Where the published fit is accurate
    # (3 <= z <= 7) it must agree with this law to the size of the next-order term.
    for z in (3.0, 4.0, 5.0, 6.0, 7.0):
        law = math.sqrt(3.0) * math.exp(-z) / math.sqrt(math.pi * z)
        assert O.ad_pvalue(z, 10 ** 9) == pytest.approx(law, rel=0.04)


def test_cdf_of_codes_and_positions():
    L = 4 * math.pi
    u = np.array([0, 1, 2 ** 31, 2 ** 32 - 1], dtype=np.uint32)
    F = O.ad_cdf_of_codes(u)
    assert np.all((F > 0) & (F < 1))
    assert F[0] == 0.5 / 2 ** 32 and F[-1] == 1 - 0.5 / 2 ** 32
    x = I.from_fixed(u, L)
    for k in range(u.size):
        assert O.ad_cdf_of_position(x[k], L) == F[k]


def test_update_rule_scripted_sequence():
    thr = 0.01
    lpth = 0.0  # start
    # (p, expected optimise, expected p_th after the step)
    script = [(0.5, False, 0.02), (0.015, False, 0.02), (0.009, True, 0.009), (0.005, False, 0.009),
              (0.004, True, 0.004), (0.03, False, 0.02), (0.0099, True, 0.0099), (0.02, False, 0.0099),
              (0.0201, False, 0.02), (0.0101, False, 0.02), (1e-300, True, 1e-300)]
    for p, opt, after in script:
        o, lpth = O.ad_schedule_step(math.log(p), thr, lpth)
        assert o == opt and lpth == pytest.approx(math.log(after), rel=1e-12), (p, o, math.exp(lpth))
    # the first step starts from p_th = 2 threshold
    o, lpth = O.ad_schedule_step(math.log(0.0101), thr, 0.0)
    assert not o and lpth == pytest.approx(math.log(0.02))
    o, lpth = O.ad_schedule_step(math.log(0.0099), thr, 0.0)
    assert o


def test_pic_run_ad_uniform_start_never_optimises():
    # quiet uniform start: the test never rejects uniformity, the width stays the caller's
    L, N, Ng = 4 * math.pi, 2048, 64
    x = I.from_fixed(I.to_fixed(I.quiet_positions(N, L, 0.0), L), L)
    v = np.zeros(N)
    cand = I.log_candidates(1.0, 1e3, 8)
    r = O.pic_run_ad(x, v, L, Ng, 0.1, 5, 50.0, cand)
    assert not r["optimised"].any()
    assert np.all(r["kappa"] == 50.0) and np.all(r["log_pvalue"] > math.log(0.9))
    ref = O.pic_run(x, v, L, Ng, 0.1, 5, kappa_u=50.0)
    np.testing.assert_array_equal(r["energy"], ref["energy"])
    np.testing.assert_array_equal(r["x"], ref["x"])


def test_pic_run_ad_non_uniform_start_and_smoothing():
    L, N, Ng = 4 * math.pi, 1024, 64
    u, v = I.landau_load(3, N, L, 0.4, 1.0)
    x = I.from_fixed(u, L)
    cand = I.log_candidates(1.0, 1e3, 12)
    rate = 0.05
    r = O.pic_run_ad(x, v, L, Ng, 0.1, 12, 5.0, cand, rate=rate)
    # strongly non-uniform: optimised at step 0, width = the CV argmin (first optimum not smoothed)
    assert r["optimised"][0] and r["log_pvalue"][0] < math.log(1e-6)
    cv0 = O.cv_curve(x, L, cand, fourier=True)
    assert r["kappa"][0] == pytest.approx(cand[O.argmin(cv0)], rel=1e-12)
    # between optimisations h = kappa^{-1/2} relaxes geometrically towards the last target
    h = r["kappa"] ** -0.5
    ht = r["h_target"]
    last_opt = np.flatnonzero(r["optimised"])[-1]
    for n in range(last_opt + 1, 12):
        assert h[n] == pytest.approx(rate * ht + (1 - rate) * h[n - 1], rel=1e-12)
