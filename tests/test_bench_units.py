"""The bench's count of algorithmic CV work against brute force."""
import math

import numpy as np

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
