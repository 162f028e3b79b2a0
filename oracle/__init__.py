"""FP64 CPU oracle for the KDE-PIC hot path -- TEST INFRASTRUCTURE ONLY.

Only the test suite, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  It shares no code with the CUDA path:
the arithmetic lives in `kde_oracle.c` (plain C, double precision, OpenMP over
independent outer loops), compiled here with gcc into `oracle/lib/`.

Every function cites the passage of the paper (Wu & Qin, arXiv 1804.11174)
that it follows; see the comments in `kde_oracle.c`.  All functions take
float64 numpy arrays; positions are float64 in [0, L).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kde_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "libkdeoracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.c_double
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, OpenMP) into oracle/lib."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            sig = {
                "or_i0e": (_D, [_D]),
                "or_vm_kernel": (_D, [_D, _D]),
                "or_bessel_ratios": (None, [_D, _I, _P]),
                "or_deposit": (None, [_P, _P, _D, _P, _I64, _I, _D, _P]),
                "or_gather": (None, [_P, _P, _D, _I64, _P, _I, _D, _P]),
                "or_poisson_spectral": (None, [_P, _I, _D, _P]),
                "or_poisson_fd": (None, [_P, _I, _D, _P]),
                "or_push": (None, [_P, _P, _P, _I64, _D, _D, _D, _D]),
                "or_field_energy": (_D, [_P, _I, _D]),
                "or_cv_dense": (_D, [_P, _P, _D, _I64, _D, _P, _P, _P]),
                "or_fourier_modes": (_I, [_D]),
                "or_cv_fourier": (_D, [_P, _I64, _D, _D, _P, _P, _P]),
                "or_cv_no_loo": (_D, [_P, _I64, _D, _D]),
                "or_adapt_widths": (None, [_P, _I64, _D, _D, _D, _D, _D, _P]),
                "or_argmin": (_I, [_P, _I]),
                "or_pic_run": (_I, [_P, _P, _P, _I, _D, _I64, _I, _D, _D, _D, _D, _D, _I, _I, _I,
                                    _P, _I, _D, _D, _D, _I, _I, _P, _P]),
                "or_damping_rate": (_I, [_P, _I, _D, _P, _P, _P]),
                "or_kde_at": (None, [_P, _P, _D, _P, _I64, _D, _P, _I64, _P]),
                "or_ad_statistic": (_D, [_P, _I64]),
                "or_bspline": (_D, [_I, _D]),
                "or_deposit_bspline": (None, [_P, _I64, _I, _D, _I, _D, _P]),
                "or_gather_bspline": (None, [_P, _I64, _I, _D, _P, _I, _D, _P]),
                "or_cv_cic": (_D, [_P, _I64, _D, _D]),
                "or_pic_run_bspline": (_I, [_P, _P, _I64, _I, _D, _I, _D, _D, _D, _D, _D, _I, _I, _P]),
                "or_ad_cdf_of_position": (_D, [_D, _D]),
                "or_ad_cdf": (_D, [_D, _I64]),
                "or_ad_pvalue": (_D, [_D, _I64]),
                "or_ad_log_pvalue": (_D, [_D, _I64]),
                "or_ad_schedule_step": (_I, [_D, _D, _P]),
                "or_pic_run_ad": (_I, [_P, _P, _P, _I64, _I, _D, _D, _D, _D, _D, _I, _I, _P, _I, _D, _D,
                                       _I, _I64, _P, _P, _P, _P, _P, _P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


def i0e(x: float) -> float:
    """exp(-x) I0(x) (Sec. II.A normalisation, scaled)."""
    return _load().or_i0e(float(x))


def vm_kernel(kappa: float, t) -> np.ndarray:
    """K_kappa(t) = e^{kappa cos t} / (2 pi I0(kappa)) (Eq. vonMises, mu = 0)."""
    lib = _load()
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    return np.array([lib.or_vm_kernel(float(kappa), float(v)) for v in t])


def bessel_ratios(kappa: float, M: int) -> np.ndarray:
    """A_m(kappa) = I_m(kappa)/I_0(kappa), m = 0..M (Fourier coefficients of the kernel)."""
    out = np.empty(M + 1, dtype=np.float64)
    _load().or_bessel_ratios(float(kappa), int(M), _ptr(out))
    return out


def deposit(x, Ng: int, L: float, kappa=None, kappa_u: float = 0.0, w=None) -> np.ndarray:
    """rho_g = sum_i w_i (2pi/L) K_{kappa_i}(theta_g - theta_i) (Eq. kde at the grid nodes)."""
    x = _f64(x)
    k = None if kappa is None else _f64(kappa)
    ww = None if w is None else _f64(w)
    rho = np.empty(Ng, dtype=np.float64)
    _load().or_deposit(_ptr(x), _ptr(k), float(kappa_u), _ptr(ww), x.size, int(Ng), float(L), _ptr(rho))
    return rho


def kde_at(x, xp, L: float, kappa=None, kappa_u: float = 0.0, w=None) -> np.ndarray:
    """The deposit's density (Eq. kde, x units) at arbitrary points xp."""
    x = _f64(x)
    xp = _f64(xp)
    k = None if kappa is None else _f64(kappa)
    ww = None if w is None else _f64(w)
    out = np.empty(xp.size, dtype=np.float64)
    _load().or_kde_at(_ptr(x), _ptr(k), float(kappa_u), _ptr(ww), x.size, float(L), _ptr(xp), xp.size, _ptr(out))
    return out


def gather(x, E, L: float, kappa=None, kappa_u: float = 0.0) -> np.ndarray:
    """E_i = sum_g (2pi/Ng) K_{kappa_i}(theta_g - theta_i) E_g."""
    x = _f64(x)
    E = _f64(E)
    k = None if kappa is None else _f64(kappa)
    out = np.empty(x.size, dtype=np.float64)
    _load().or_gather(_ptr(x), _ptr(k), float(kappa_u), x.size, _ptr(E), E.size, float(L), _ptr(out))
    return out


def poisson(rho_total, L: float, fd: bool = False) -> np.ndarray:
    """E from dE/dx = rho_total: spectral (E_m = rho_m/(i k_m)) or the paper's FD scheme."""
    r = _f64(rho_total)
    E = np.empty(r.size, dtype=np.float64)
    lib = _load()
    (lib.or_poisson_fd if fd else lib.or_poisson_spectral)(_ptr(r), r.size, float(L), _ptr(E))
    return E


def push(x, v, Ei, L: float, dt: float, qm: float, kick: float = 1.0):
    """Leap-frog push (Sec. III.A); returns new (x, v)."""
    x = _f64(x).copy()
    v = _f64(v).copy()
    Ei = _f64(Ei)
    _load().or_push(_ptr(x), _ptr(v), _ptr(Ei), x.size, float(L), float(dt), float(qm), float(kick))
    return x, v


def field_energy(E, L: float) -> float:
    E = _f64(E)
    return _load().or_field_energy(_ptr(E), E.size, float(L))


def cv_dense(x, L: float, kappa=None, kappa_u: float = 0.0, want_loo: bool = False):
    """Eq. (cv_def), dense pairs; returns (cv, int_f2, pair_mean, loo or None), x units."""
    x = _f64(x)
    k = None if kappa is None else _f64(kappa)
    loo = np.empty(x.size, dtype=np.float64) if want_loo else None
    f2 = ctypes.c_double()
    pm = ctypes.c_double()
    cv = _load().or_cv_dense(_ptr(x), _ptr(k), float(kappa_u), x.size, float(L), _ptr(loo),
                             ctypes.addressof(f2), ctypes.addressof(pm))
    return cv, f2.value, pm.value, loo


def fourier_modes(kappa: float) -> int:
    return _load().or_fourier_modes(float(kappa))


def cv_fourier(x, L: float, kappa: float, want_loo: bool = False):
    """Eq. (cv_def) for a uniform width in exact Fourier form; same returns as cv_dense."""
    x = _f64(x)
    loo = np.empty(x.size, dtype=np.float64) if want_loo else None
    f2 = ctypes.c_double()
    pm = ctypes.c_double()
    cv = _load().or_cv_fourier(_ptr(x), x.size, float(L), float(kappa), _ptr(loo),
                               ctypes.addressof(f2), ctypes.addressof(pm))
    return cv, f2.value, pm.value, loo


def cv_curve(x, L: float, cands, kappa_rel=None, fourier: bool = False) -> np.ndarray:
    """CV(kappa_c) for every candidate.  With kappa_rel the candidates are scale factors
    applied to per-particle widths (dense pairs only)."""
    out = []
    for c in cands:
        if kappa_rel is not None:
            out.append(cv_dense(x, L, kappa=float(c) * _f64(kappa_rel))[0])
        elif fourier:
            out.append(cv_fourier(x, L, float(c))[0])
        else:
            out.append(cv_dense(x, L, kappa_u=float(c))[0])
    return np.array(out)


def cv_no_loo(x, L: float, kappa: float) -> float:
    """Appendix A: the CV function without leave-one-out (x units)."""
    x = _f64(x)
    return _load().or_cv_no_loo(_ptr(x), x.size, float(L), float(kappa))


def adapt_widths(loo, L: float, kappa_star: float, alpha: float = 0.5,
                 kmin: float = 0.0, kmax: float = 1e300) -> np.ndarray:
    """Silverman particle-wise widths (Sec. II.C) from leave-one-out densities (x units)."""
    loo = _f64(loo)
    out = np.empty(loo.size, dtype=np.float64)
    _load().or_adapt_widths(_ptr(loo), loo.size, float(L), float(kappa_star), float(alpha),
                            float(kmin), float(kmax), _ptr(out))
    return out


def argmin(cv) -> int:
    cv = _f64(cv)
    return _load().or_argmin(_ptr(cv), cv.size)


def pic_run(x, v, L: float, Ng: int, dt: float, nsteps: int, kappa=None, kappa_u: float = 0.0,
            qm: float = -1.0, charge: float = -1.0, background: float = 1.0, fd: bool = False,
            width_every: int = 0, cands=None, alpha: float = 0.5, kmin: float = 0.0,
            kmax: float = 1e300, cv_fourier_form: bool = True, backstep: bool = True):
    """Electrostatic PIC run (Sec. III.A) with KDE deposit; returns dict with x, v, kappa,
    energy W[n] and kappa*[n]."""
    x = _f64(x).copy()
    v = _f64(v).copy()
    N = x.size
    kap = _f64(kappa).copy() if kappa is not None else np.zeros(N)
    cand = _f64(cands) if cands is not None else np.zeros(1)
    W = np.empty(nsteps, dtype=np.float64)
    ks = np.empty(nsteps, dtype=np.float64)
    _load().or_pic_run(_ptr(x), _ptr(v), _ptr(kap), int(kappa is not None), float(kappa_u), N,
                       int(Ng), float(L), float(dt), float(qm), float(charge), float(background),
                       int(fd), int(nsteps), int(width_every), _ptr(cand),
                       int(cand.size if cands is not None else 0), float(alpha), float(kmin),
                       float(kmax), int(cv_fourier_form), int(backstep), _ptr(W), _ptr(ks))
    return {"x": x, "v": v, "kappa": kap if kappa is not None else None, "energy": W, "kstar": ks}


def damping_rate(W, dt: float):
    """Amplitude damping rate from the first two maxima of ln W after t = 0 (Sec. III.B)."""
    W = _f64(W)
    g = ctypes.c_double()
    p1 = ctypes.c_int()
    p2 = ctypes.c_int()
    rc = _load().or_damping_rate(_ptr(W), W.size, float(dt), ctypes.addressof(g),
                                 ctypes.addressof(p1), ctypes.addressof(p2))
    if rc != 0:
        raise ValueError("fewer than two energy maxima")
    return g.value, p1.value, p2.value


def ad_statistic(F) -> float:
    """Anderson-Darling A^2 of CDF values F(X_i) in (0, 1) against the uniform (Sec. II.D)."""
    F = _f64(F)
    return _load().or_ad_statistic(_ptr(F), F.size)


def ad_cdf_of_codes(u):
    """The uniform CDF as the test sees 32-bit position codes: (u + 1/2) / 2^32."""
    return (np.asarray(u, dtype=np.uint32).astype(np.float64) + 0.5) / 4294967296.0


def ad_cdf_of_position(x: float, L: float) -> float:
    return _load().or_ad_cdf_of_position(float(x), float(L))


def ad_cdf(z: float, n: int) -> float:
    """P(A^2 <= z) for n uniform samples (Marsaglia & Marsaglia 2004)."""
    return _load().or_ad_cdf(float(z), int(n))


def ad_pvalue(a2: float, n: int) -> float:
    """p-value of A^2 for n samples (Marsaglia up to A^2 = 7, the limiting tail beyond)."""
    return _load().or_ad_pvalue(float(a2), int(n))


def ad_log_pvalue(a2: float, n: int) -> float:
    return _load().or_ad_log_pvalue(float(a2), int(n))


def ad_schedule_step(lp: float, threshold: float, lp_th: float):
    """One step of the Sec. II.D update rule on ln p-values; lp_th >= 0 means "start".
    Returns (optimise, new lp_th)."""
    s = ctypes.c_double(lp_th)
    r = _load().or_ad_schedule_step(float(lp), float(threshold), ctypes.addressof(s))
    return bool(r), s.value


def pic_run_ad(x, v, L: float, Ng: int, dt: float, nsteps: int, kappa_u: float, cands,
               threshold: float = 0.01, rate: float = 0.05, qm: float = -1.0, charge: float = -1.0,
               background: float = 1.0, fd: bool = False, backstep: bool = True, step0: int = 0,
               lp_th: float = 0.0, h_target: float = 0.0):
    """Electrostatic PIC run (Sec. III.A) whose uniform width follows the Anderson-Darling
    update algorithm of Sec. II.D; returns dict with x, v, the state (kappa, p_th, h_target)
    and per-step energy, kappa, ln p-value and optimisation flags."""
    x = _f64(x).copy()
    v = _f64(v).copy()
    cand = _f64(cands)
    k = ctypes.c_double(kappa_u)
    pth = ctypes.c_double(lp_th)
    ht = ctypes.c_double(h_target)
    W = np.empty(nsteps, dtype=np.float64)
    ks = np.empty(nsteps, dtype=np.float64)
    pv = np.empty(nsteps, dtype=np.float64)
    cvf = np.empty(nsteps, dtype=np.int32)
    _load().or_pic_run_ad(_ptr(x), _ptr(v), ctypes.addressof(k), x.size, int(Ng), float(L), float(dt),
                          float(qm), float(charge), float(background), int(fd), int(nsteps), _ptr(cand),
                          cand.size, float(threshold), float(rate), int(backstep), int(step0),
                          ctypes.addressof(pth), ctypes.addressof(ht), _ptr(W), _ptr(ks), _ptr(pv),
                          _ptr(cvf))
    return {"x": x, "v": v, "kappa_u": k.value, "lp_th": pth.value, "h_target": ht.value, "energy": W,
            "kappa": ks, "log_pvalue": pv, "optimised": cvf.astype(bool)}


def bspline(p: int, t) -> np.ndarray:
    """Centred cardinal B-spline of degree p (Cox-de Boor recursion), support |t| < (p+1)/2."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    f = _load().or_bspline
    return np.array([f(int(p), float(v)) for v in t])


def deposit_bspline(x, Ng: int, L: float, order: int, h: float) -> np.ndarray:
    """Standard-PIC deposit with the B-spline shape of degree `order` and width h (x units)."""
    x = _f64(x)
    rho = np.empty(Ng, dtype=np.float64)
    _load().or_deposit_bspline(_ptr(x), x.size, int(order), float(h), int(Ng), float(L), _ptr(rho))
    return rho


def gather_bspline(x, E, L: float, order: int, h: float) -> np.ndarray:
    x = _f64(x)
    E = _f64(E)
    out = np.empty(x.size, dtype=np.float64)
    _load().or_gather_bspline(_ptr(x), x.size, int(order), float(h), _ptr(E), E.size, float(L), _ptr(out))
    return out


def cv_cic(x, L: float, h: float) -> float:
    """CV of the first-order (CIC) shape of width h (x units)."""
    x = _f64(x)
    return _load().or_cv_cic(_ptr(x), x.size, float(L), float(h))


def pic_run_bspline(x, v, L: float, Ng: int, dt: float, nsteps: int, order: int = 1, h: float = 0.0,
                    qm: float = -1.0, charge: float = -1.0, background: float = 1.0, backstep: bool = True):
    """Standard PIC run with the B-spline shape of degree `order` and width h (0: dx); spectral
    Poisson; returns dict with x, v and the field energy W[n]."""
    x = _f64(x).copy()
    v = _f64(v).copy()
    h = h if h > 0 else L / Ng
    W = np.empty(nsteps, dtype=np.float64)
    _load().or_pic_run_bspline(_ptr(x), _ptr(v), x.size, int(order), float(h), int(Ng), float(L), float(dt),
                               float(qm), float(charge), float(background), int(nsteps), int(backstep), _ptr(W))
    return {"x": x, "v": v, "energy": W}
