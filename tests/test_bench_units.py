"""The bench's counts of algorithmic work (CV pairs, deposit and gather window pairs) against brute force,
and its Landau root solver against the textbook root."""
import math

import numpy as np
import pytest

import kde_inputs as I


def test_inradius_pair_count_matches_brute_force():
    from bench import cv_inradius_pairs
    u = I.cv_sweep_load(3, 700)
    th = u.astype(np.float64) * (2 * math.pi / 2 ** 32)
    d = np.abs(th[:, None] - th[None, :])
    d = np.minimum(d, 2 * math.pi - d)
    iu = np.triu_indices(th.size, 1)
    for k in [1.0, 9.0, 100.0, 1e4]:
        s2 = 24 * math.log(2) / (2 * k)
        r = math.pi if s2 >= 1 else 2 * math.asin(math.sqrt(s2))
        brute = int(np.sum(d[iu] <= r))
        assert cv_inradius_pairs(u, [k]) == brute


def test_window_pair_count_matches_node_counts():
    # the deposit/gather roofline unit: nodes within the truncation radius of a particle,
    # averaged over positions, equals 2 r Ng / (2 pi) (whole grid once r >= pi)
    from bench import grid_window_pairs
    rng = np.random.default_rng(5)
    Ng = 256
    th = rng.uniform(0, 2 * math.pi, 20000)
    g = 2 * math.pi * np.arange(Ng) / Ng
    for k in [4.0, 12.0, 100.0, 3000.0]:
        s2 = min(24 * math.log(2) / (2 * k), 1.0)
        r = 2 * math.asin(math.sqrt(s2))
        d = np.abs(th[:, None] - g[None, :])
        d = np.minimum(d, 2 * math.pi - d)
        counts = np.sum(d <= r, axis=1)
        est = grid_window_pairs(np.full(th.size, k), Ng)
        assert abs(counts.sum() - est) <= 0.01 * est + th.size * 1e-6


def test_landau_theory_root():
    # the bench's kinetic Langmuir root: k lambda_D = 0.5 gives omega = 1.41566 - 0.15336 i
    # (textbook value); the statistics workload (k = 1) uses the same solver with a
    # smoothing factor F of mode k, which lowers omega_p^2 by F^2 and changes the rate
    from bench import landau_theory
    assert landau_theory(1.0, k=0.5) == pytest.approx(-0.15336, abs=2e-5)
    assert landau_theory(2.0, k=0.25) == pytest.approx(-0.15336, abs=2e-5)  # depends on k v_th only
    g1, g2 = landau_theory(0.4, k=1.0), landau_theory(0.4, k=1.0, factor=0.98)
    assert math.isfinite(g1) and math.isfinite(g2) and g1 != g2


def test_clock_samples_kept_for_the_timed_region():
    # the sampler's summary from stamped nvidia-smi lines (fields: sm, max sm, power,
    # active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap)
    from bench import ClockSampler

    def line(sm, cap="Not Active", hw="Not Active"):
        return "%d, 2070, 900.0, 0x0, %s, Not Active, Not Active, %s" % (sm, hw, cap)

    lines = [(0.00, line(1200)), (0.05, line(2070)), (0.10, line(2070, cap="Active")),
             (0.15, line(2055)), (0.20, line(900, hw="Active")), (0.25, "garbled")]
    s = ClockSampler.summarise(lines, 0.04, 0.16)
    assert s["window"] == "timed region" and s["samples"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["reasons"] == ["sw_power_cap"]
    # a region between two samples: the neighbours on either side
    s = ClockSampler.summarise(lines, 0.16, 0.17)
    assert s["window"] == "nearest to the timed region" and s["samples"] == 2
    assert s["reasons"] == ["hw_slowdown"]
    # no marks: every sample
    s = ClockSampler.summarise(lines)
    assert s["window"] == "whole run" and s["samples"] == 5
    assert ClockSampler.summarise([(0.0, "garbled")]) is None
