"""Pins of the oracle's standard-PIC shapes (B-splines of degree 1, 2, 3, 5; the comparison of
Sec. IV) against facts that do not come from the oracle: unit integral, partition of unity,
tabulated values, the convolution identity behind the CIC width CV, exact charge conservation
of the standard deposit, exact interpolation of a constant field, and CV by brute-force
quadrature on tiny samples."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 7])
def test_unit_integral_and_symmetry(p):
    half = (p + 1) / 2
    knots = np.arange(-half, half + 1e-9, 1.0)
    total = sum(integrate.quad(lambda t: O.bspline(p, t)[0], a, b, epsabs=1e-13)[0]
                for a, b in zip(knots[:-1], knots[1:]))
    assert total == pytest.approx(1.0, abs=1e-11)
    t = np.linspace(-half - 0.5, half + 0.5, 41)
    np.testing.assert_allclose(O.bspline(p, t), O.bspline(p, -t), atol=1e-15)
    assert np.all(O.bspline(p, np.array([-half - 0.01, half + 0.01])) == 0.0)


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_partition_of_unity(p):
    rng = np.random.default_rng(p)
    for t in rng.random(10):
        ks = np.arange(-8, 9)
        assert O.bspline(p, t - ks).sum() == pytest.approx(1.0, abs=1e-13)


def test_tabulated_values():
    assert O.bspline(1, 0.0)[0] == 1.0 and O.bspline(1, 0.5)[0] == 0.5
    assert O.bspline(2, 0.0)[0] == pytest.approx(0.75) and O.bspline(2, 1.0)[0] == pytest.approx(0.125)
    assert O.bspline(3, 0.0)[0] == pytest.approx(2 / 3) and O.bspline(3, 1.0)[0] == pytest.approx(1 / 6)
    assert O.bspline(5, 0.0)[0] == pytest.approx(11 / 20) and O.bspline(5, 1.0)[0] == pytest.approx(13 / 60)
    assert O.bspline(5, 2.0)[0] == pytest.approx(1 / 120)


def test_cic_autoconvolution_is_cubic():
    # (B_1 * B_1)(t) = int B_1(s) B_1(t - s) ds = B_3(t): the identity the CIC width CV uses
    for t in (0.0, 0.3, 0.9, 1.0, 1.4, 1.99, 2.5):
        c = integrate.quad(lambda s: O.bspline(1, s)[0] * O.bspline(1, t - s)[0], -1, 1,
                           points=[0.0, t - 1, t, t + 1], epsabs=1e-14)[0]
        assert c == pytest.approx(O.bspline(3, t)[0], abs=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_standard_deposit_conserves_charge_and_gather_is_exact(p):
    L, Ng, N = 2 * math.pi, 64, 257
    rng = np.random.default_rng(10 + p)
    x = rng.random(N) * L
    dx = L / Ng
    rho = O.deposit_bspline(x, Ng, L, p, dx)
    assert rho.sum() * dx == pytest.approx(L, rel=1e-13)
    E = O.gather_bspline(x, np.full(Ng, 0.37), L, p, dx)
    np.testing.assert_allclose(E, 0.37, rtol=1e-13)
    # wider shapes conserve charge only up to aliasing but integrate to the same total in the mean
    rho2 = O.deposit_bspline(x, Ng, L, p, 2.5 * dx)
    assert rho2.sum() * dx == pytest.approx(L, rel=1e-2)


def test_cic_single_particle_at_a_node():
    L, Ng = 2 * math.pi, 32
    dx = L / Ng
    rho = O.deposit_bspline(np.array([5 * dx]), Ng, L, 1, dx)
    expect = np.zeros(Ng)
    expect[5] = L / dx
    np.testing.assert_allclose(rho, expect, atol=1e-12)


def test_cv_cic_by_quadrature():
    # int fhat^2 of the piecewise-linear estimate by quadrature between its kinks
    L, h = 2 * math.pi, 0.4
    rng = np.random.default_rng(5)
    for N in (2, 3, 5):
        x = rng.random(N) * L
        n = N

        def fhat(t):
            d = (t - x + L / 2) % L - L / 2
            return np.sum(np.maximum(0.0, 1.0 - np.abs(d) / h)) / (n * h)

        kinks = np.sort(np.concatenate([(x + k * h) % L for k in (-1, 0, 1)]))
        pts = np.concatenate([[0.0], kinks, [L]])
        f2 = sum(integrate.quad(lambda t: fhat(t) ** 2, a, b, epsabs=1e-14)[0] for a, b in zip(pts[:-1], pts[1:]))
        pair = 0.0
        for i in range(N):
            for j in range(N):
                if i != j:
                    d = (x[i] - x[j] + L / 2) % L - L / 2
                    pair += max(0.0, 1.0 - abs(d) / h) / h
        ref = f2 - 2.0 * pair / (n * (n - 1))
        assert O.cv_cic(x, L, h) == pytest.approx(ref, rel=1e-10, abs=1e-13)
