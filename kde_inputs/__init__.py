"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module holds no arithmetic of the KDE method itself: it only draws
particle loads (positions, velocities, widths) and candidate grids.  Both the
product path and the oracle consume exactly the arrays produced here, so any
difference between them comes from the method's arithmetic alone ("common
random numbers", Sec. III.B of the paper).

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: value(seed, stream, k) = mix(key(seed, stream) + (k + 1) * GAMMA).

Positions are returned both as float64 in [0, L) and as the periodic 32-bit
fixed-point code u = floor(x / L * 2**32) that the CUDA path stores; the oracle
is always fed x = u * L / 2**32 so both sides see the same points.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
TWO32 = 4294967296.0

# stream identifiers: one independent counter stream per drawn quantity
STREAM_X, STREAM_V1, STREAM_V2, STREAM_MIX, STREAM_VM, STREAM_KAPPA, STREAM_REQ = range(1, 8)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """`count` 64-bit outputs of the counter-based SplitMix64 stream (seed, stream)."""
    with np.errstate(over="ignore"):
        key = _mix(np.array([(seed * 0x100000001B3 + stream * 0x9E3779B1) & 0xFFFFFFFFFFFFFFFF],
                            dtype=np.uint64))[0]
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        return _mix(key + k * GAMMA)


def uniforms(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits each."""
    return (splitmix64(seed, stream, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def to_fixed(x: np.ndarray, L: float) -> np.ndarray:
    """Periodic 32-bit fixed-point code of positions x in [0, L)."""
    t = np.mod(np.asarray(x, dtype=np.float64) / L, 1.0) * TWO32
    return np.minimum(np.floor(t), TWO32 - 1).astype(np.uint32)


def from_fixed(u: np.ndarray, L: float) -> np.ndarray:
    """Exact float64 position of each 32-bit code."""
    return np.asarray(u, dtype=np.float64) * (L / TWO32)


def inverse_cdf_cosine(q: np.ndarray, L: float, alpha: float, mode: int = 1) -> np.ndarray:
    """Solve F(x) = q on [0, L) for the density (1 + alpha*cos(k x))/L, k = 2*pi*mode/L.

    F(x) = (x + alpha/k * sin(k x)) / L is strictly increasing for |alpha| < 1;
    Newton's method from x = q L converges to machine precision.
    """
    q = np.asarray(q, dtype=np.float64)
    if abs(alpha) >= 1.0:
        raise ValueError("|alpha| must be < 1")
    if alpha == 0.0:
        return q * L
    k = 2.0 * math.pi * mode / L
    x = q * L
    for _ in range(100):
        f = (x + (alpha / k) * np.sin(k * x)) / L - q
        step = f / ((1.0 + alpha * np.cos(k * x)) / L)
        x = x - step
        if np.max(np.abs(step)) < 1e-15 * L:
            break
    return np.mod(x, L)


def quiet_positions(N: int, L: float, alpha: float, mode: int = 1) -> np.ndarray:
    """Quiet start: x_j = F^{-1}((j + 1/2) / N)."""
    return inverse_cdf_cosine((np.arange(N, dtype=np.float64) + 0.5) / N, L, alpha, mode)


def random_positions(seed: int, N: int, L: float, alpha: float, mode: int = 1) -> np.ndarray:
    """Independent draws from (1 + alpha cos(2 pi mode x / L)) / L by inverse CDF."""
    return inverse_cdf_cosine(uniforms(seed, STREAM_X, N), L, alpha, mode)


def maxwellian(seed: int, N: int, vth: float) -> np.ndarray:
    """Box-Muller normal draws with standard deviation vth."""
    u1 = 1.0 - uniforms(seed, STREAM_V1, N)          # (0, 1]
    u2 = uniforms(seed, STREAM_V2, N)
    return vth * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def von_mises_draws(seed: int, N: int, mu: float, kappa: float) -> np.ndarray:
    """Von Mises(mu, kappa) angles in [0, 2 pi) by the Best & Fisher (1979) rejection method."""
    tau = 1.0 + math.sqrt(1.0 + 4.0 * kappa * kappa)
    rho = (tau - math.sqrt(2.0 * tau)) / (2.0 * kappa)
    r = (1.0 + rho * rho) / (2.0 * rho)
    out = np.empty(N, dtype=np.float64)
    todo = np.arange(N)
    attempt = 0
    while todo.size:
        draw = uniforms(seed, STREAM_VM, 3 * N, attempt * 3 * N)
        u1 = draw[0::3][todo]
        u2 = draw[1::3][todo]
        u3 = draw[2::3][todo]
        z = np.cos(math.pi * u1)
        f = (1.0 + r * z) / (r + z)
        c = kappa * (r - f)
        u2 = np.maximum(u2, 1e-300)
        ok = (c * (2.0 - c) - u2 > 0.0) | (np.log(c / u2) + 1.0 - c >= 0.0)
        th = mu + np.sign(u3 - 0.5) * np.arccos(np.clip(f, -1.0, 1.0))
        out[todo[ok]] = np.mod(th[ok], 2.0 * math.pi)
        todo = todo[~ok]
        attempt += 1
        if attempt > 200:
            raise RuntimeError("von Mises rejection sampler did not terminate")
    return out


def mixture_angles(seed: int, N: int, w_uniform: float = 0.7, mu: float = math.pi,
                   kappa: float = 20.0) -> np.ndarray:
    """Angles in [0, 2 pi) from w_uniform * U[0, 2pi) + (1 - w_uniform) * vonMises(mu, kappa)."""
    pick = uniforms(seed, STREAM_MIX, N)
    uni = 2.0 * math.pi * uniforms(seed, STREAM_X, N)
    vm = von_mises_draws(seed, N, mu, kappa)
    return np.where(pick < w_uniform, uni, vm)


def log_uniform(seed: int, stream: int, N: int, lo: float, hi: float) -> np.ndarray:
    """Log-uniform draws in [lo, hi]."""
    return lo * np.exp(uniforms(seed, stream, N) * math.log(hi / lo))


def log_candidates(lo: float, hi: float, n: int) -> np.ndarray:
    """n log-spaced widths kappa_c = lo * (hi/lo)**(c/(n-1)), c = 0..n-1."""
    if n == 1:
        return np.array([lo], dtype=np.float64)
    return lo * (hi / lo) ** (np.arange(n, dtype=np.float64) / (n - 1))


# ---------------------------------------------------------------------------
# workload recipes (sizes and distributions of the paper's Langmuir / Landau
# runs and of the CV sweep); each returns plain numpy arrays
# ---------------------------------------------------------------------------

def langmuir_load(N: int = 4096, L: float = 4 * math.pi, alpha: float = 0.01):
    """Cold Langmuir wave: quiet start of 1 + alpha cos(2 pi x / L), v = 0."""
    x = quiet_positions(N, L, alpha)
    u = to_fixed(x, L)
    return u, np.zeros(N, dtype=np.float64)


def landau_load(seed: int, N: int, L: float = 4 * math.pi, alpha: float = 0.05, vth: float = 1.0):
    """Landau damping load: random inverse-CDF positions and Maxwellian velocities."""
    u = to_fixed(random_positions(seed, N, L, alpha), L)
    v = maxwellian(seed, N, vth)
    return u, v


def landau_quiet_load(N: int, L: float = 4 * math.pi, alpha: float = 0.05, vth: float = 1.0):
    """Low-noise Landau load: quiet positions, velocities by the normal quantile of a
    bit-reversed (van der Corput) sequence so position and velocity are uncorrelated."""
    from scipy.special import ndtri
    u = to_fixed(quiet_positions(N, L, alpha), L)
    j = np.arange(N, dtype=np.uint64)
    rev = np.zeros(N, dtype=np.float64)
    scale = 0.5
    jj = j.copy()
    while np.any(jj):
        rev += (jj & np.uint64(1)).astype(np.float64) * scale
        jj >>= np.uint64(1)
        scale *= 0.5
    v = vth * ndtri(np.clip(rev + 0.5 / N, 1e-16, 1 - 1e-16))
    return u, v


def cv_sweep_load(seed: int, N: int = 1 << 18):
    """CV sweep positions on [0, 2 pi): 0.7 uniform + 0.3 von Mises(pi, 20)."""
    L = 2 * math.pi
    return to_fixed(mixture_angles(seed, N), L)


def ensemble_sizes(n_real: int = 256, seed: int = 0):
    """Per-realisation particle counts N_r = round(2**(14 + 6 U_r)) and grids Ng_r cycling
    through {128, 256, 512, 1024}."""
    Ns = np.rint(2.0 ** (14.0 + 6.0 * uniforms(seed, STREAM_REQ, n_real))).astype(np.int64)
    Ngs = np.array([128, 256, 512, 1024], dtype=np.int64)[np.arange(n_real) % 4]
    return Ns, Ngs
