"""Pins for the oracle's cross-validation (Sec. II.B, Eq. cv_def), Appendix A and the
particle-wise widths (Sec. II.C).

* Three independent evaluations of CV agree: dense pairs with the closed-form
  two-fold convolution, the exact Fourier form, and (for the integral term)
  brute-force quadrature of fhat^2 built from SciPy's Bessel function.
* Unbiasedness (Sec. II.B): E[CV(kappa)] + int f^2 = MISE(kappa), with the exact
  MISE of the von Mises KDE for a known truth, checked over many realisations.
* Appendix A: without leave-one-out the CV decreases towards kappa -> infinity.
* Silverman widths: evenly spaced samples give lambda_i = 1; the geometric mean of
  lambda_i is 1.
"""
import math

import numpy as np
import pytest
import scipy.special as sp

import kde_inputs as I


def vm_numpy(k, t):
    # independent evaluation of the kernel through SciPy's scaled Bessel function
    return np.exp(k * (np.cos(t) - 1.0)) / (2 * math.pi * sp.i0e(k))


@pytest.mark.parametrize("k", [0.8, 15.0, 250.0, 4000.0])
def test_dense_and_fourier_agree(oracle, k):
    L = 4 * math.pi
    x = I.from_fixed(I.to_fixed(I.mixture_angles(1, 300) * L / (2 * math.pi), L), L)
    d = oracle.cv_dense(x, L, kappa_u=k, want_loo=True)
    f = oracle.cv_fourier(x, L, k, want_loo=True)
    assert d[0] == pytest.approx(f[0], rel=1e-12, abs=1e-14)
    assert d[1] == pytest.approx(f[1], rel=1e-12)
    assert d[2] == pytest.approx(f[2], rel=1e-12)
    np.testing.assert_allclose(d[3], f[3], rtol=1e-10, atol=1e-13)
    # the leave-one-out densities average to the pair term
    assert d[3].mean() == pytest.approx(d[2], rel=1e-13)


@pytest.mark.parametrize("kind", ["uniform", "per-particle"])
def test_integral_term_by_quadrature(oracle, kind):
    # int fhat^2 by brute-force quadrature on a fine grid, independent of the
    # closed-form two-fold convolution the oracle uses
    L = 2 * math.pi
    n = 12
    x = I.uniforms(3, 1, n) * L
    if kind == "uniform":
        kap = np.full(n, 37.0)
    else:
        kap = I.log_uniform(3, 6, n, 2.0, 400.0)
    M = 1 << 16
    t = np.arange(M) * (2 * math.pi / M)
    f = np.zeros(M)
    for j in range(n):
        f += vm_numpy(kap[j], t - x[j]) / n
    quad = (2 * math.pi / M) * np.sum(f * f)
    cv, f2, pm, _ = oracle.cv_dense(x, L, kappa=kap)
    assert f2 == pytest.approx(quad, rel=1e-11)


def test_tiny_brute_force(oracle):
    # N = 5, per-particle widths: the leave-one-out term by direct enumeration
    L = 3.0
    x = np.array([0.1, 0.4, 1.7, 2.2, 2.95])
    kap = np.array([3.0, 10.0, 0.5, 80.0, 7.0])
    n = len(x)
    th = 2 * math.pi * x / L
    loo = np.zeros(n)
    for i in range(n):
        for j in range(n):
            if i != j:
                loo[i] += vm_numpy(kap[j], th[i] - th[j])
    loo *= (2 * math.pi / L) / (n - 1)
    cv, f2, pm, loo_o = oracle.cv_dense(x, L, kappa=kap, want_loo=True)
    np.testing.assert_allclose(loo_o, loo, rtol=1e-13)
    assert pm == pytest.approx(loo.mean(), rel=1e-13)
    assert cv == pytest.approx(f2 - 2 * pm, rel=1e-13)


def mixture_phi(m):
    # characteristic function (theta units) of 0.7 U + 0.3 vonMises(pi, 20)
    m = np.asarray(m)
    return np.where(m == 0, 1.0, 0.3 * (sp.ive(m, 20.0) / sp.ive(0, 20.0)) * (-1.0) ** m)


def exact_mise(k, n, M=400):
    m = np.arange(1, M + 1)
    Am = sp.ive(m, k) / sp.ive(0, k)
    p2 = mixture_phi(m) ** 2
    return (1 / math.pi) * np.sum((Am - 1) ** 2 * p2 + Am ** 2 * (1 - p2) / n)


def int_f2_truth(M=400):
    m = np.arange(1, M + 1)
    return (1 / (2 * math.pi)) * (1 + 2 * np.sum(mixture_phi(m) ** 2))


def test_cv_is_unbiased_for_mise(oracle):
    # Sec. II.B: CV(h) + int f^2 is an unbiased estimator of MISE(h)
    L = 2 * math.pi
    n = 48
    R = 400
    ks = [3.0, 20.0, 150.0]
    vals = np.zeros((R, len(ks)))
    for r in range(R):
        x = I.mixture_angles(1000 + r, n)
        for c, k in enumerate(ks):
            vals[r, c] = oracle.cv_fourier(x, L, k)[0]
    f2 = int_f2_truth()
    for c, k in enumerate(ks):
        mean = vals[:, c].mean()
        se = vals[:, c].std(ddof=1) / math.sqrt(R)
        assert abs(mean + f2 - exact_mise(k, n)) < 5 * se, (k, mean + f2, exact_mise(k, n), se)
    # and the estimator is informative: mean CV orders the widths like the exact MISE
    order_cv = np.argsort(vals.mean(axis=0))
    order_mise = np.argsort([exact_mise(k, n) for k in ks])
    assert list(order_cv) == list(order_mise)


def test_mixture_truth_constants():
    # int f^2 of the CV-sweep mixture (theta units)
    assert int_f2_truth() == pytest.approx(0.25728, abs=5e-5)


def test_appendix_a_no_loo_prefers_zero_width(oracle):
    L = 2 * math.pi
    x = I.mixture_angles(5, 200)
    ks = I.log_candidates(10.0, 1e6, 12)
    no_loo = [oracle.cv_no_loo(x, L, k) for k in ks]
    assert all(b < a for a, b in zip(no_loo, no_loo[1:]))
    loo = [oracle.cv_fourier(x, L, k)[0] for k in ks]
    assert int(np.argmin(loo)) < len(ks) - 1  # the leave-one-out CV has an interior minimum


def test_argmin_smallest_index_on_ties(oracle):
    assert oracle.argmin([3.0, 1.0, 2.0, 1.0]) == 1


def test_adaptive_widths_uniform_samples(oracle):
    L = 4 * math.pi
    n = 64
    x = (np.arange(n) + 0.25) * L / n
    _, _, _, loo = oracle.cv_dense(x, L, kappa_u=50.0, want_loo=True)
    k = oracle.adapt_widths(loo, L, 50.0, 0.5)
    np.testing.assert_allclose(k, 50.0, rtol=1e-12)


def test_adaptive_widths_geometric_mean_and_order(oracle):
    L = 2 * math.pi
    x = I.mixture_angles(9, 400)
    kstar = 60.0
    _, _, _, loo = oracle.cv_dense(x, L, kappa_u=kstar, want_loo=True)
    k = oracle.adapt_widths(loo, L, kstar, 0.5)
    # prod lambda_i = 1  =>  mean log kappa_i = log kappa*
    assert np.mean(np.log(k)) == pytest.approx(math.log(kstar), rel=1e-12)
    # denser regions get narrower kernels (larger kappa)
    n = len(x)
    K0 = (2 * math.pi / L) / (2 * math.pi * sp.i0e(kstar))
    ft = ((n - 1) * loo + K0) / n
    assert np.all(np.diff(k[np.argsort(ft)]) >= -1e-9)
    # alpha = 0 leaves every width at kappa*
    np.testing.assert_allclose(oracle.adapt_widths(loo, L, kstar, 0.0), kstar, rtol=1e-14)
    # clamping
    kc = oracle.adapt_widths(loo, L, kstar, 0.5, kmin=55.0, kmax=65.0)
    assert kc.min() >= 55.0 and kc.max() <= 65.0


def _two_cluster_sample(n_dense=48, n_sparse=5):
    # a tight cluster around theta = 1 plus a few isolated points: the isolated points'
    # leave-one-out densities are far below their own kernel's peak, so the pilot with
    # and without the self term differ by orders of magnitude there
    th_dense = 1.0 + 0.08 * (I.uniforms(21, 0, n_dense) - 0.5)
    th_sparse = 2.0 + (2 * math.pi - 2.5) * (np.arange(n_sparse) + 0.5) / n_sparse
    return np.concatenate([th_dense, th_sparse])


def _pilot_full_kde(th, kstar, L):
    # pilot estimate f~(X_i): the KDE at kappa* evaluated at X_i over all n samples,
    # its own kernel included (x units), by direct summation with SciPy's i0e
    d = th[:, None] - th[None, :]
    K = np.exp(kstar * (np.cos(d) - 1.0)) / (2 * math.pi * sp.i0e(kstar))
    return (2 * math.pi / L) * K.mean(axis=1)


def _loo_direct(th, kstar, L):
    n = th.size
    d = th[:, None] - th[None, :]
    K = np.exp(kstar * (np.cos(d) - 1.0)) / (2 * math.pi * sp.i0e(kstar))
    np.fill_diagonal(K, 0.0)
    return (2 * math.pi / L) * K.sum(axis=1) / (n - 1)


@pytest.mark.parametrize("alpha", [0.5, 0.3])
def test_adaptive_widths_pilot_includes_self_term(oracle, alpha):
    # Sec. II.C with Silverman's pilot: lambda_i = (f~(X_i)/g)^(-alpha), g the geometric
    # mean of f~, h_i = h lambda_i, kappa = 1/h^2.  The pilot here is the full KDE at X_i
    # computed directly (not from the leave-one-out sums); the reading without the self
    # term must fail on this sample.
    L = 4 * math.pi
    th = _two_cluster_sample()
    kstar = 300.0
    loo = _loo_direct(th, kstar, L)
    k = oracle.adapt_widths(loo, L, kstar, alpha)
    ft = _pilot_full_kde(th, kstar, L)
    lam = np.exp(-alpha * (np.log(ft) - np.mean(np.log(ft))))
    np.testing.assert_allclose(k, kstar / lam ** 2, rtol=1e-10)
    lam_no_self = np.exp(-alpha * (np.log(loo) - np.mean(np.log(loo))))
    assert np.max(np.abs(kstar / lam_no_self ** 2 / k - 1.0)) > 0.5


def test_adaptive_widths_scale_the_kernel_width_by_lambda(oracle):
    # h_i = h lambda_i (Sec. II.C) measured on the kernels themselves: the circular
    # standard deviation sqrt(2 (1 - A_1(kappa))) of a von Mises kernel is
    # kappa^(-1/2) (1 + O(1/kappa)), so the ratio of kernel widths must equal lambda_i
    # to O(1/kappa).  A_1 from SciPy's ive.  Mapping kappa_i = kappa*/lambda_i (an h^2
    # scaling) would give sqrt(lambda_i) instead.
    L = 2 * math.pi
    th = _two_cluster_sample(64, 6)
    kstar = 2500.0
    loo = _loo_direct(th, kstar, L)
    k = oracle.adapt_widths(loo, L, kstar, 0.5)
    ft = _pilot_full_kde(th, kstar, L)
    lam = (ft / np.exp(np.mean(np.log(ft)))) ** -0.5
    assert lam.max() / lam.min() > 4.0                   # the sample spans a wide range
    A1 = lambda kk: sp.ive(1, kk) / sp.ive(0, kk)
    width = np.sqrt(2 * (1 - A1(k)))
    width_star = math.sqrt(2 * (1 - A1(kstar)))
    rel = width / width_star / lam - 1.0
    assert np.max(np.abs(rel)) < 0.5 / k.min()
