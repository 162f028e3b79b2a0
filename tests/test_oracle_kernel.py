"""Pins for the oracle's von Mises kernel and Bessel functions (Sec. II.A, Eq. vonMises).

The oracle is checked against things it does not compute itself: SciPy's
scaled Bessel routines (special cases that reduce to a library routine), the
normalisation integral by brute-force quadrature, and the Gaussian limit
1/kappa ~ sigma^2 stated in Sec. II.A.
"""
import math

import numpy as np
import pytest
import scipy.special as sp

KAPPAS = [0.05, 0.7, 1.0, 8.0, 29.9, 30.0, 30.5, 100.0, 1e3, 1e4, 1e5]


@pytest.mark.parametrize("k", KAPPAS)
def test_i0e_matches_library(oracle, k):
    assert oracle.i0e(k) == pytest.approx(sp.i0e(k), rel=2e-15)


def test_i0_textbook_value(oracle):
    # I0(1) = 1.266065877752008 (Abramowitz & Stegun, Table 9.8)
    assert oracle.i0e(1.0) * math.e == pytest.approx(1.266065877752008, rel=1e-14)


@pytest.mark.parametrize("k", [0.3, 1.0, 10.0, 100.0, 1e3, 1e4])
def test_kernel_integrates_to_one(oracle, k):
    # int_0^{2pi} K = 1 (first consistency condition of Sec. II.B).  K is even, so
    # integrate over [0, pi] with the trapezoid rule (spectrally accurate: the
    # integrand is smooth and its odd derivatives vanish at both ends).
    m = 20_001
    tt = np.linspace(0.0, math.pi, m)
    KK = oracle.vm_kernel(k, tt)
    h = tt[1] - tt[0]
    integral = 2.0 * h * (KK.sum() - 0.5 * (KK[0] + KK[-1]))
    assert integral == pytest.approx(1.0, rel=1e-10)


@pytest.mark.parametrize("k", [0.5, 4.0, 40.0, 400.0])
def test_kernel_fourier_modes(oracle, k):
    # int K(t) cos(m t) dt = I_m(kappa) / I_0(kappa)
    m_max = 6
    n = 4096
    t = np.arange(n) * (2 * math.pi / n)
    K = oracle.vm_kernel(k, t)
    for m in range(m_max + 1):
        c = (2 * math.pi / n) * np.sum(K * np.cos(m * t))
        assert c == pytest.approx(sp.ive(m, k) / sp.ive(0, k), rel=1e-10, abs=1e-14)


def test_kernel_symmetric_and_peaked(oracle):
    t = np.linspace(0.01, 3.1, 50)
    for k in [1.0, 50.0]:
        a = oracle.vm_kernel(k, t)
        b = oracle.vm_kernel(k, -t)
        np.testing.assert_allclose(a, b, rtol=1e-15)
        assert np.all(oracle.vm_kernel(k, [0.0])[0] > a)


def test_kernel_gaussian_limit(oracle):
    # Sec. II.A: 1/kappa plays the role of sigma^2; for large kappa the kernel tends to
    # the normal density with that variance near its centre
    k = 1e5
    s = 1.0 / math.sqrt(k)
    t = np.linspace(-2 * s, 2 * s, 9)
    gauss = np.exp(-t * t / (2 * s * s)) / (s * math.sqrt(2 * math.pi))
    np.testing.assert_allclose(oracle.vm_kernel(k, t), gauss, rtol=2e-5)


@pytest.mark.parametrize("k", [0.2, 3.0, 30.0, 500.0, 1e4])
def test_bessel_ratios_match_library(oracle, k):
    M = 80
    A = oracle.bessel_ratios(k, M)
    ref = sp.ive(np.arange(M + 1), k) / sp.ive(0, k)
    mask = ref > 1e-250
    np.testing.assert_allclose(A[mask], ref[mask], rtol=1e-12)


def test_fourier_mode_cutoff(oracle):
    for k in [1.0, 100.0, 1e4]:
        M = oracle.fourier_modes(k)
        A = sp.ive(np.arange(M + 2), k) / sp.ive(0, k)
        assert A[M] < 1e-17
        assert A[M - 1] >= 1e-18 * 0.999
