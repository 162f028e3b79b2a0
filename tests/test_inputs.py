"""The seeded input generators: determinism, distributions and the fixed-point code."""
import math

import numpy as np
import pytest
import scipy.stats as st

import kde_inputs as I


def test_determinism_and_streams():
    a = I.uniforms(7, 1, 1000)
    b = I.uniforms(7, 1, 1000)
    c = I.uniforms(7, 2, 1000)
    d = I.uniforms(8, 1, 1000)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c) and not np.array_equal(a, d)
    # offsets continue the same stream
    np.testing.assert_array_equal(I.uniforms(7, 1, 500, 500), a[500:])
    assert a.min() >= 0.0 and a.max() < 1.0


def test_uniformity():
    u = I.uniforms(1, 1, 200_000)
    assert st.kstest(u, "uniform").pvalue > 1e-4


def test_inverse_cdf_solves_cdf():
    L = 4 * math.pi
    q = I.uniforms(2, 1, 1000)
    x = I.inverse_cdf_cosine(q, L, 0.05)
    k = 2 * math.pi / L
    F = (x + 0.05 / k * np.sin(k * x)) / L
    np.testing.assert_allclose(F, q, atol=1e-13)


def test_random_positions_follow_density():
    L = 4 * math.pi
    x = I.random_positions(0, 400_000, L, 0.3)
    k = 2 * math.pi / L
    cdf = lambda t: (t + 0.3 / k * np.sin(k * t)) / L
    assert st.kstest(x, cdf).pvalue > 1e-4


def test_maxwellian():
    v = I.maxwellian(3, 200_000, 1.0)
    assert st.kstest(v, "norm").pvalue > 1e-4


def test_von_mises_sampler():
    th = I.von_mises_draws(4, 100_000, math.pi, 20.0)
    assert st.kstest(th, st.vonmises(20.0, loc=math.pi).cdf).pvalue > 1e-4


def test_fixed_point_roundtrip():
    L = 4 * math.pi
    x = I.uniforms(9, 1, 10_000) * L
    u = I.to_fixed(x, L)
    assert u.dtype == np.uint32
    err = x - I.from_fixed(u, L)
    assert err.min() >= 0.0 and err.max() < L / 2 ** 32 * 1.0001


def test_candidate_grid():
    c = I.log_candidates(1.0, 1e3, 16)
    assert c[0] == 1.0 and c[-1] == pytest.approx(1e3)
    np.testing.assert_allclose(np.diff(np.log10(c)), 3 / 15)


def test_ensemble_sizes():
    Ns, Ngs = I.ensemble_sizes(256)
    assert Ns.min() >= 2 ** 14 and Ns.max() <= 2 ** 20
    assert set(Ngs.tolist()) == {128, 256, 512, 1024}
