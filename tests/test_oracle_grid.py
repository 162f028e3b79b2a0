"""Pins for the oracle's deposit (Eq. kde at the nodes), gather, Poisson solves and push.

Closed forms used (derived from the Fourier series K(t) = (1/2pi) sum_m A_m e^{imt},
A_m = I_m/I_0 taken from SciPy):
  * one particle: the grid DFT of rho is (w Ng / L) sum_{n = m mod Ng} A_n e^{-i n theta_i};
  * N evenly spaced particles: rho(theta) = 1 + 2 sum_{p>=1} A_{pN} cos(pN (theta - phi));
  * a single cosine charge density gives E = (alpha/k) sin(kx) (spectral) and
    alpha (dx/2) cot(k dx / 2) sin(kx) (the paper's finite-difference scheme);
  * gathering cos(m theta_g) gives A_m cos(m theta_i) plus grid aliases.
"""
import math

import numpy as np
import pytest
import scipy.special as sp

import kde_inputs as I


def A(n, k):
    n = np.abs(np.asarray(n))
    return sp.ive(n, k) / sp.ive(0, k)


@pytest.mark.parametrize("k,Ng", [(3.0, 16), (40.0, 32), (500.0, 24)])
def test_single_particle_grid_dft(oracle, k, Ng):
    L = 4 * math.pi
    x = np.array([1.2345])
    w = np.array([0.7])
    rho = oracle.deposit(x, Ng, L, kappa_u=k, w=w)
    th = 2 * math.pi * x[0] / L
    dft = np.fft.fft(rho)
    for m in range(Ng):
        n = m + Ng * np.arange(-60, 61)
        ref = (w[0] * Ng / L) * np.sum(A(n, k) * np.exp(-1j * n * th))
        assert abs(dft[m] - ref) < 1e-11 * max(1.0, abs(ref))


@pytest.mark.parametrize("k,N", [(2.0, 5), (30.0, 12), (300.0, 40)])
def test_evenly_spaced_particles(oracle, k, N):
    L = 2.0
    phi = 0.37
    x = (np.arange(N) / N + phi / (2 * math.pi)) * L
    Ng = 50
    rho = oracle.deposit(x, Ng, L, kappa_u=k)
    tg = 2 * math.pi * np.arange(Ng) / Ng
    ref = np.ones(Ng)
    for p in range(1, 40):
        ref += 2 * A(p * N, k) * np.cos(p * N * (tg - phi))
    np.testing.assert_allclose(rho, ref, rtol=1e-12, atol=1e-13)


def test_charge_conservation_within_aliasing(oracle):
    L = 4 * math.pi
    Ng = 64
    u, _ = I.landau_load(3, 500, L)
    x = I.from_fixed(u, L)
    for k in [1.0, 10.0, 100.0]:
        rho = oracle.deposit(x, Ng, L, kappa_u=k)
        total = rho.sum() * L / Ng
        bound = 2 * sum(A(p * Ng, k) for p in range(1, 10)) * L
        assert abs(total - L) <= bound + 1e-12


def test_per_particle_widths_are_superposition(oracle):
    L = 1.0
    x = np.array([0.1, 0.55, 0.9])
    k = np.array([5.0, 50.0, 500.0])
    w = np.array([0.2, 0.3, 0.5])
    Ng = 40
    tot = oracle.deposit(x, Ng, L, kappa=k, w=w)
    parts = sum(oracle.deposit(x[i:i + 1], Ng, L, kappa_u=k[i], w=w[i:i + 1]) for i in range(3))
    np.testing.assert_allclose(tot, parts, rtol=1e-14)


@pytest.mark.parametrize("Ng", [16, 33, 64])
def test_poisson_single_mode(oracle, Ng):
    L = 4 * math.pi
    k = 2 * math.pi / L * 3
    xg = np.arange(Ng) * L / Ng
    rho = 0.05 * np.cos(k * xg) + 0.8  # a constant part is removed by the solve
    E = oracle.poisson(rho, L)
    np.testing.assert_allclose(E, 0.05 / k * np.sin(k * xg), atol=1e-13)
    dx = L / Ng
    Efd = oracle.poisson(rho, L, fd=True)
    ref = 0.05 * (dx / 2) / math.tan(k * dx / 2) * np.sin(k * xg)
    np.testing.assert_allclose(Efd, ref, atol=1e-12)


def test_poisson_fd_satisfies_difference_equations(oracle):
    L = 3.0
    Ng = 40
    rng = I.uniforms(11, 1, Ng)
    rho = rng - rng.mean()
    E = oracle.poisson(rho, L, fd=True)
    dx = L / Ng
    # Fourier symbol of the FD scheme, derived from the two difference equations:
    # phi_m = rho_m dx^2 / (4 sin^2(pi m/Ng)), E_m = -i sin(2 pi m/Ng)/dx phi_m,
    # i.e. E_m = rho_m / (i (2/dx) tan(pi m / Ng)); the oracle solves in real space.
    rm = np.fft.fft(rho)
    em = np.fft.fft(E)
    for m in range(1, Ng):
        if 2 * m == Ng:
            assert abs(em[m]) < 1e-12
            continue
        ms = m if 2 * m < Ng else m - Ng
        sym = 1j * (2 / dx) * math.tan(math.pi * ms / Ng)
        assert abs(em[m] - rm[m] / sym) < 1e-11


def test_poisson_spectral_derivative_gives_back_rho(oracle):
    L = 5.0
    Ng = 32
    r = I.uniforms(5, 2, Ng)
    rho = r - r.mean()
    E = oracle.poisson(rho, L)
    k = 2 * math.pi * np.fft.fftfreq(Ng, d=L / Ng)
    dE = np.real(np.fft.ifft(1j * k * np.fft.fft(E)))
    rm = np.fft.fft(rho)
    rm[Ng // 2] = 0.0  # the Nyquist mode is dropped by the solve
    np.testing.assert_allclose(dE, np.real(np.fft.ifft(rm)), atol=1e-12)


@pytest.mark.parametrize("k", [2.0, 60.0])
def test_gather_single_mode(oracle, k):
    L = 4 * math.pi
    Ng = 32
    m = 3
    tg = 2 * math.pi * np.arange(Ng) / Ng
    E = np.cos(m * tg)
    x = I.from_fixed(I.to_fixed(I.uniforms(1, 3, 50) * L, L), L)
    th = 2 * math.pi * x / L
    out = oracle.gather(x, E, L, kappa_u=k)
    ref = np.zeros_like(th)
    for p in range(-40, 41):
        for n in (m + p * Ng, -m + p * Ng):
            ref += 0.5 * A(n, k) * np.cos(n * th)
    np.testing.assert_allclose(out, ref, atol=1e-12)


def test_gather_constant_field(oracle):
    L = 1.0
    Ng = 128
    x = I.uniforms(2, 3, 40) * L
    out = oracle.gather(x, np.full(Ng, 2.5), L, kappa_u=20.0)
    np.testing.assert_allclose(out, 2.5, rtol=1e-13)


def test_total_force_vanishes_uniform_width(oracle):
    # deposit, spectral solve and gather with one kernel conserve momentum:
    # sum_i E_i = dx * sum_g E_g rho_e,g = 0 because sum_g E_g rho_total,g = 0.
    L = 4 * math.pi
    Ng = 64
    u, _ = I.landau_load(7, 2000, L)
    x = I.from_fixed(u, L)
    rho = oracle.deposit(x, Ng, L, kappa_u=80.0)
    E = oracle.poisson(1.0 - rho, L)
    Ei = oracle.gather(x, E, L, kappa_u=80.0)
    assert abs(Ei.sum()) < 1e-12 * np.abs(Ei).sum()


def test_push_leapfrog(oracle):
    L = 2.0
    x = np.array([0.1, 1.95])
    v = np.array([1.0, 0.5])
    Ei = np.array([0.2, -0.4])
    xn, vn = oracle.push(x, v, Ei, L, dt=0.1, qm=-1.0, kick=0.5)
    np.testing.assert_allclose(vn, [1.0 - 0.5 * 0.2 * 0.1, 0.5 + 0.5 * 0.4 * 0.1])
    np.testing.assert_allclose(xn, np.mod(x + vn * 0.1, L))


@pytest.mark.parametrize("Ng", [8, 37, 256])
def test_field_energy_single_sine_closed_form(oracle, Ng):
    # W = 1/2 sum_g E_g^2 dx (Sec. III.B).  For E_g = a sin(2 pi m g / Ng) with
    # 0 < m < Ng/2, sum_g sin^2 = Ng/2, so W = a^2 L / 4 exactly; a constant field c
    # gives W = c^2 L / 2.
    L = 4 * math.pi
    a = 0.37
    g = np.arange(Ng)
    for m in (1, 3):
        E = a * np.sin(2 * math.pi * m * g / Ng)
        assert oracle.field_energy(E, L) == pytest.approx(a * a * L / 4, rel=1e-13)
    assert oracle.field_energy(np.full(Ng, 1.5), L) == pytest.approx(1.5 * 1.5 * L / 2, rel=1e-14)


def test_field_energy_exchanges_with_kinetic_energy(oracle):
    # Cold Langmuir oscillation: with deposit and gather through one kernel,
    # d/dt (1/2 int E^2 dx) = sum_i w v_i E_i = -d/dt (1/2 sum_i w v_i^2)
    # (Ampere's law dE/dt = -J from continuity and Gauss's law), so the field energy
    # reported by the oracle plus the kinetic energy of the electrons (mass w = L/N
    # each, q/m = -1) stays at its t = 0 value, when all of it sits in the field.
    # A dropped 1/2 or dx in the field energy breaks the balance by a factor >= 2.
    L = 4 * math.pi
    N, Ng, kappa, dt = 4096, 64, 10.0, 0.05
    x = I.from_fixed(I.to_fixed(I.quiet_positions(N, L, 0.01), L), L)
    v = np.zeros(N)
    w = L / N

    def field_at(xx):
        rho = oracle.deposit(xx, Ng, L, kappa_u=kappa)
        E = oracle.poisson(1.0 - rho, L)
        return E, oracle.gather(xx, E, L, kappa_u=kappa)

    E, Ei = field_at(x)
    W0 = oracle.field_energy(E, L)
    assert W0 > 0
    x, v = oracle.push(x, v, Ei, L, dt, -1.0, kick=0.5)   # v^{1/2}, x^1
    ke_prev = 0.5 * w * float(np.sum(v * v))
    totals, kes = [], []
    for _ in range(140):                                  # ~ one plasma period
        E, Ei = field_at(x)
        Wf = oracle.field_energy(E, L)
        x, v = oracle.push(x, v, Ei, L, dt, -1.0)
        ke = 0.5 * w * float(np.sum(v * v))
        totals.append(Wf + 0.5 * (ke_prev + ke))
        kes.append(ke)
        ke_prev = ke
    totals = np.array(totals)
    assert np.max(np.abs(totals - W0)) < 0.005 * W0
    assert max(kes) == pytest.approx(W0, rel=0.005)


def test_kde_at_single_particle(oracle):
    # Eq. (kde) for one particle of weight w: (2 pi / L) w K_kappa(theta_p - theta_1),
    # the von Mises density.  Normalisation from SciPy (i0e; the vonmises
    # distribution for moderate widths), not the oracle's own Bessel function.
    import scipy.stats as st
    L = 4 * math.pi
    x1 = np.array([2.3])
    xp = np.linspace(0.0, L, 53, endpoint=False) + 0.011
    dth = 2 * math.pi * (xp - x1[0]) / L
    for k in (0.5, 7.0, 40.0, 3000.0):
        out = oracle.kde_at(x1, xp, L, kappa_u=k, w=np.array([1.7]))
        ref = (2 * math.pi / L) * 1.7 * np.exp(k * (np.cos(dth) - 1.0)) / (2 * math.pi * sp.i0e(k))
        np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-300)
        if k <= 40.0:
            ref2 = (2 * math.pi / L) * 1.7 * st.vonmises.pdf(dth, k)
            np.testing.assert_allclose(out, ref2, rtol=1e-9)
    # default weight L/N with N = 1 is L
    out = oracle.kde_at(x1, xp, L, kappa_u=7.0)
    np.testing.assert_allclose(out, 2 * math.pi * np.exp(7.0 * (np.cos(dth) - 1.0)) / (2 * math.pi * sp.i0e(7.0)),
                               rtol=1e-12)


@pytest.mark.parametrize("k,N", [(3.0, 5), (45.0, 16), (900.0, 96)])
def test_kde_at_evenly_spaced_between_nodes(oracle, k, N):
    # N evenly spaced particles, default weights L/N: the KDE is the Fourier series
    # 1 + 2 sum_p A_pN(kappa) cos(pN (theta - phi)) everywhere, evaluated here at
    # random points that are not grid nodes.
    L = 3.0
    phi = 1.1
    x = (np.arange(N) / N + phi / (2 * math.pi)) * L
    xp = I.uniforms(11, 0, 41) * L
    out = oracle.kde_at(x, xp, L, kappa_u=k)
    th = 2 * math.pi * xp / L
    ref = np.ones_like(th)
    for p in range(1, 60):
        ref += 2 * A(p * N, k) * np.cos(p * N * (th - phi))
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-13)


def test_kde_at_per_particle_widths_superpose(oracle):
    L = 2.0
    x = np.array([0.2, 0.9, 1.7])
    kap = np.array([4.0, 250.0, 60.0])
    w = np.array([0.5, 1.25, 2.0])
    xp = I.uniforms(12, 0, 29) * L
    out = oracle.kde_at(x, xp, L, kappa=kap, w=w)
    ref = np.zeros_like(xp)
    for xi, ki, wi in zip(x, kap, w):
        d = 2 * math.pi * (xp - xi) / L
        ref += (2 * math.pi / L) * wi * np.exp(ki * (np.cos(d) - 1.0)) / (2 * math.pi * sp.i0e(ki))
    np.testing.assert_allclose(out, ref, rtol=1e-12)
