"""GB300 (sm_103a) KDE particle-in-cell hot path: thin Python binding of libkdepic.

Method: Wu & Qin, "Reducing Noise for PIC Simulations Using Kernel Density
Estimation Algorithm" (arXiv 1804.11174).  Every computation runs in the CUDA
kernels of `libkdepic.so` behind the C ABI of `include/kdepic.h`; this module
only marshals arguments (torch tensors supply device memory and streams) and
turns status codes into exceptions.  There is no CPU fallback: if the library
is missing, importing the binding raises.

Function names follow the C entry points: `Context.deposit` calls
`kde_deposit`, `Context.cv` calls `kde_cv`, `Context.pic_step` calls
`pic_step`, and so on.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

from . import _build

__all__ = ["Context", "PicState", "Server", "Ensemble", "KdeError", "load_library", "LIB_PATH", "F64", "POISSON_FD", "CV_SCALE", "CV_SPECTRAL", "CV_PAIRS",
           "PIC_NO_BACKSTEP", "MAX_NG"]

LIB_PATH = _build.LIB
F64 = 0x1
POISSON_FD = 0x2
CV_SCALE = 0x4
CV_SPECTRAL = 0x8
CV_PAIRS = 0x10
PIC_NO_BACKSTEP = 0x100
MAX_NG = 4096

_P = ctypes.c_void_p
_D = ctypes.c_double
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_U32 = ctypes.c_uint32


class KdeError(RuntimeError):
    """A libkdepic call returned a non-zero status."""

    def __init__(self, name, code, msg):
        super().__init__("%s failed with status %d: %s" % (name, code, msg))
        self.code = code


class _PicState(ctypes.Structure):
    _fields_ = [
        ("u", _P), ("v", _P), ("kappa", _P), ("kappa_norm", _P), ("id", _P),
        ("N", _I64), ("Ng", _I32),
        ("L", _D), ("dt", _D), ("qm", _D), ("charge", _D), ("background", _D), ("kappa_uniform", _D),
        ("width_every", _I32), ("cand", _P), ("n_cand", _I32),
        ("alpha", _D), ("kappa_min", _D), ("kappa_max", _D),
        ("energy", _P), ("kappa_star", _P), ("step", _I64), ("flags", _U32),
        ("width_ad", _I32), ("ad_threshold", _D), ("adjust_rate", _D), ("ad_log_pth", _D), ("h_target", _D),
        ("n_opt", _I64), ("ad_log_p", _P), ("shape_order", _I32), ("shape_h", _D),
    ]


class _Request(ctypes.Structure):
    _fields_ = [
        ("kind", _I32), ("N", _I64), ("Ng", _I32), ("L", _D), ("u", _P), ("kappa", _P), ("kappa_uniform", _D),
        ("v", _P), ("field", _P), ("cand", _P), ("n_cand", _I32), ("n_steps", _I32), ("dt", _D), ("out", _P),
        ("out64", _P), ("out_argmin", _P), ("flags", _U32),
    ]


REQ_DEPOSIT, REQ_GATHER, REQ_CV, REQ_PIC = 1, 2, 3, 4

_lib = None


def load_library(path: str | None = None):
    """Load libkdepic.so (build it first with `__graft_entry__.build()`)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError("libkdepic.so not found at %s: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')" % p)
    lib = ctypes.CDLL(p)
    S = ctypes.c_int
    sigs = {
        "kde_create": (S, [ctypes.POINTER(_P), ctypes.c_int, _P]),
        "kde_destroy": (S, [_P]),
        "kde_set_stream": (S, [_P, _P]),
        "kde_last_error": (ctypes.c_char_p, [_P]),
        "kde_sync": (S, [_P]),
        "kde_reserve": (S, [_P, _I64, _I32, _I32]),
        "kde_pack_positions": (S, [_P, _P, _I64, _D, _P]),
        "kde_deposit": (S, [_P, _P, _P, _D, _P, _I64, _I32, _D, _P, _U32]),
        "kde_poisson": (S, [_P, _P, _I32, _D, _D, _D, _P, _P, _U32]),
        "kde_gather": (S, [_P, _P, _P, _D, _I64, _P, _I32, _D, _P, _U32]),
        "kde_cv": (S, [_P, _P, _P, _I64, _D, _P, _I32, _P, _P, _P, _U32]),
        "kde_ad_test": (S, [_P, _P, _I64, _P, _P]),
        "kde_deposit_bspline": (S, [_P, _P, _I64, _I32, _D, _I32, _D, _P]),
        "kde_gather_bspline": (S, [_P, _P, _I64, _I32, _D, _P, _I32, _D, _P]),
        "kde_cv_cic": (S, [_P, _P, _I64, _D, _P, _I32, _P, _P]),
        "kde_ensemble_create": (S, [_P, ctypes.POINTER(_P), _I32, _P, _P, _P, _D, _D, _P, _P]),
        "kde_ensemble_set_widths": (S, [_P, _P]),
        "kde_ensemble_set_shape": (S, [_P, _I32, _D]),
        "kde_ensemble_mise": (S, [_P, _D, _I32, _P]),
        "kde_ensemble_run": (S, [_P, _I32, _P, _I32]),
        "kde_ensemble_destroy": (S, [_P]),
        "kde_adapt_widths": (S, [_P, _P, _I64, _D, _D, _D, _D, _D, _P]),
        "pic_step": (S, [_P, ctypes.POINTER(_PicState), _I32]),
        "pic_step_host": (S, [_P, ctypes.POINTER(_PicState), _I32]),
        "kde_damping_rate": (S, [_P, _I64, _D, _P]),
        "kde_probe_exp2": (S, [_P, _I64, _P, _P]),
        "kde_probe_fma": (S, [_P, _I64, _P, _P]),
        "kde_profile_enable": (S, [_P, ctypes.c_int]),
        "kde_deposit_noalloc": (S, [_P, _P, _P, _D, _P, _I64, _I32, _D, _P, _U32]),
        "kde_server_create": (S, [ctypes.POINTER(_P), ctypes.c_int, _I32, _I64]),
        "kde_server_submit": (S, [_P, ctypes.POINTER(_Request), ctypes.POINTER(_I64)]),
        "kde_server_wait": (S, [_P, _I64, _P, _P]),
        "kde_server_wait_times": (S, [_P, _I64, _P]),
        "kde_server_wait_msg": (S, [_P, _I64, _P, ctypes.c_char_p, ctypes.c_int32]),
        "kde_server_cancel": (S, [_P, _I64]),
        "kde_server_stats": (S, [_P, _P]),
        "kde_server_destroy": (S, [_P]),
        "kde_profile_read": (S, [_P, ctypes.c_int, _P, _P]),
        "kde_set_autotune": (S, [_P, ctypes.c_int32]),
        "kde_set_launch_overlap": (S, [_P, ctypes.c_int32]),
        "kde_set_truncation": (S, [_P, ctypes.c_double]),
        "kde_autotune_table": (S, [_P, ctypes.c_int32, _P, _P, _P, _P]),
        "kde_autotune_set": (S, [_P, ctypes.c_int32, _P, _P, _P]),
        "kde_set_wait_limit": (S, [_P, _I64]),
        "kde_autotune_entries": (S, [_P, _P]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _ptr(t):
    if t is None:
        return None
    return t.data_ptr()


def _torch():
    import torch
    return torch


class Context:
    """One kde_ctx bound to a CUDA device and stream (default: torch's current stream)."""

    def __init__(self, device: int = 0, stream=None):
        torch = _torch()
        self.lib = load_library()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = _P()
        rc = self.lib.kde_create(ctypes.byref(h), int(device), _P(stream.cuda_stream))
        if rc != 0:
            raise KdeError("kde_create", rc, "cannot use CUDA device %d" % device)
        self.h = h

    # -- plumbing ---------------------------------------------------------
    def _check(self, name, rc):
        if rc != 0:
            raise KdeError(name, rc, self.lib.kde_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.kde_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self.stream = stream
        self._check("kde_set_stream", self.lib.kde_set_stream(self.h, _P(stream.cuda_stream)))

    def sync(self):
        self._check("kde_sync", self.lib.kde_sync(self.h))

    def reserve(self, N: int, Ng: int, n_cand: int = 0):
        self._check("kde_reserve", self.lib.kde_reserve(self.h, int(N), int(Ng), int(n_cand)))

    def _new(self, n, dtype):
        torch = _torch()
        return torch.empty(int(n), dtype=dtype, device="cuda:%d" % self.device)

    # -- C ABI entry points -------------------------------------------------
    def pack_positions(self, x, L: float, out=None):
        torch = _torch()
        out = self._new(x.numel(), torch.int32) if out is None else out
        self._check("kde_pack_positions", self.lib.kde_pack_positions(self.h, _ptr(x), x.numel(), float(L), _ptr(out)))
        return out

    def deposit(self, u, Ng: int, L: float, kappa=None, kappa_uniform: float = 0.0, weight=None, out=None,
                dtype=None):
        """kde_deposit: rho_g = sum_i w_i (2pi/L) K_{kappa_i}(theta_g - theta_i)."""
        torch = _torch()
        dtype = dtype or (kappa.dtype if kappa is not None else torch.float32)
        out = self._new(Ng, dtype) if out is None else out
        flags = F64 if out.dtype == torch.float64 else 0
        self._check("kde_deposit", self.lib.kde_deposit(self.h, _ptr(u), _ptr(kappa), float(kappa_uniform),
                                                        _ptr(weight), u.numel(), int(Ng), float(L), _ptr(out), flags))
        return out

    def poisson(self, rho, L: float, charge: float = -1.0, background: float = 1.0, fd: bool = False, out=None,
                energy=None):
        """kde_poisson: E from dE/dx = background + charge * rho (spectral or FD)."""
        torch = _torch()
        out = self._new(rho.numel(), rho.dtype) if out is None else out
        flags = (F64 if rho.dtype == torch.float64 else 0) | (POISSON_FD if fd else 0)
        self._check("kde_poisson", self.lib.kde_poisson(self.h, _ptr(rho), rho.numel(), float(L), float(charge),
                                                        float(background), _ptr(out), _ptr(energy), flags))
        return out

    def gather(self, u, field, L: float, kappa=None, kappa_uniform: float = 0.0, out=None):
        """kde_gather: E_i = sum_g (2pi/Ng) K_{kappa_i}(theta_g - theta_i) field_g."""
        torch = _torch()
        out = self._new(u.numel(), field.dtype) if out is None else out
        flags = F64 if field.dtype == torch.float64 else 0
        self._check("kde_gather", self.lib.kde_gather(self.h, _ptr(u), _ptr(kappa), float(kappa_uniform), u.numel(),
                                                      _ptr(field), field.numel(), float(L), _ptr(out), flags))
        return out

    def cv(self, u, L: float, cand, kappa_rel=None, loo=None, want_loo: bool = False, spectral: bool = False,
           pairs: bool = False):
        """kde_cv: CV(kappa_c) (x units) for every candidate; returns (cv, argmin, loo).
        spectral=True selects the exact Fourier form, pairs=True the O(N^2) pair sums
        (uniform widths); neither: the library's cost rule picks the cheaper exact form."""
        torch = _torch()
        cand = np.ascontiguousarray(cand, dtype=np.float64)
        cv = np.empty(cand.size, dtype=np.float64)
        am = ctypes.c_int32()
        if want_loo and loo is None:
            loo = self._new(u.numel(), torch.float32)
        flags = (CV_SCALE if kappa_rel is not None else 0) | (CV_SPECTRAL if spectral else 0) | (CV_PAIRS if pairs else 0)
        self._check("kde_cv", self.lib.kde_cv(self.h, _ptr(u), _ptr(kappa_rel), u.numel(), float(L),
                                              cand.ctypes.data, cand.size, cv.ctypes.data, ctypes.addressof(am),
                                              _ptr(loo), flags))
        return cv, am.value, loo

    def deposit_bspline(self, u, Ng: int, L: float, order: int, h: float, out=None):
        """kde_deposit_bspline: standard-PIC shape of degree `order` and width h (x units)."""
        torch = _torch()
        if out is None:
            out = torch.empty(int(Ng), dtype=torch.float32, device=u.device)
        self._check("kde_deposit_bspline", self.lib.kde_deposit_bspline(self.h, _ptr(u), u.numel(), int(order),
                                                                        float(h), int(Ng), float(L), _ptr(out)))
        return out

    def gather_bspline(self, u, field, L: float, order: int, h: float, out=None):
        torch = _torch()
        if out is None:
            out = torch.empty(u.numel(), dtype=torch.float32, device=u.device)
        self._check("kde_gather_bspline", self.lib.kde_gather_bspline(self.h, _ptr(u), u.numel(), int(order),
                                                                      float(h), _ptr(field), field.numel(), float(L),
                                                                      _ptr(out)))
        return out

    def cv_cic(self, u, L: float, h_cand):
        """kde_cv_cic: CV of the CIC shape's width over candidates h (x units); returns (cv, argmin)."""
        h = np.ascontiguousarray(h_cand, dtype=np.float64)
        cv = np.empty(h.size, dtype=np.float64)
        am = ctypes.c_int32()
        self._check("kde_cv_cic", self.lib.kde_cv_cic(self.h, _ptr(u), u.numel(), float(L), h.ctypes.data, h.size,
                                                      cv.ctypes.data, ctypes.addressof(am)))
        return cv, am.value

    def ad_test(self, u):
        """Anderson-Darling test of the positions against the uniform distribution (Sec. II.D):
        returns (A^2, ln p)."""
        a2 = ctypes.c_double()
        lp = ctypes.c_double()
        self._check("kde_ad_test", self.lib.kde_ad_test(self.h, _ptr(u), u.numel(), ctypes.addressof(a2),
                                                        ctypes.addressof(lp)))
        return a2.value, lp.value

    def adapt_widths(self, loo, L: float, kappa_star: float, alpha: float = 0.5, kappa_min: float = 0.0,
                     kappa_max: float = 1e6, out=None):
        """kde_adapt_widths: Silverman particle-wise widths from leave-one-out densities."""
        torch = _torch()
        out = self._new(loo.numel(), torch.float32) if out is None else out
        self._check("kde_adapt_widths", self.lib.kde_adapt_widths(self.h, _ptr(loo), loo.numel(), float(L),
                                                                  float(kappa_star), float(alpha), float(kappa_min),
                                                                  float(kappa_max), _ptr(out)))
        return out

    def pic_step(self, state: "PicState", n_steps: int):
        """pic_step: advance the run by n_steps leap-frog steps (stream-ordered)."""
        if state.max_steps and state.c.step + int(n_steps) > state.max_steps:
            raise KdeError("pic_step", 1, "energy history holds %d steps; step %d + %d would overflow it"
                           % (state.max_steps, state.c.step, n_steps))
        state._sync_in()
        self._check("pic_step", self.lib.pic_step(self.h, ctypes.byref(state.c), int(n_steps)))

    def pic_step_host(self, state: "PicState", n_steps: int):
        """pic_step_host: pic_step on a state whose tensors live in host memory (pinned for
        DMA): the library copies it in, runs, copies it back and synchronises."""
        if state.u.is_cuda or state.v.is_cuda:
            raise KdeError("pic_step_host", 1, "the state's tensors must be host tensors")
        if state.max_steps and state.c.step + int(n_steps) > state.max_steps:
            raise KdeError("pic_step_host", 1, "history holds %d steps; step %d + %d would overflow it"
                           % (state.max_steps, state.c.step, n_steps))
        state._sync_in()
        self._check("pic_step_host", self.lib.pic_step_host(self.h, ctypes.byref(state.c), int(n_steps)))

    PROF = {"cv_pairs": 0, "deposit": 1, "gather": 2, "sort": 3, "poisson": 4, "cv_grid": 5, "cv_loo": 6,
            "spectral": 7, "ad": 8, "deposit_rows": 9}

    def set_wait_limit(self, polls: int = -1):
        """kde_set_wait_limit: polls of a bounded device wait (-1: default, 0: give up at once)."""
        self._check("kde_set_wait_limit", self.lib.kde_set_wait_limit(self.h, int(polls)))

    def set_autotune(self, on: bool = True):
        """kde_set_autotune: tune the FP32 gather's tile shape per key on first use."""
        self._check("kde_set_autotune", self.lib.kde_set_autotune(self.h, int(on)))

    def set_truncation(self, log2_cut: float = 0.0):
        """kde_set_truncation: FP32 kernels cut at 2^-log2_cut of their peak (0: default / tuned)."""
        self._check("kde_set_truncation", self.lib.kde_set_truncation(self.h, float(log2_cut)))

    def autotune_table(self):
        """kde_autotune_table: every stored autotuner choice as a dict with the key's grid
        size, log2 N and width class (0: per-particle widths, else 4 log2(kappa) + 128),
        the kind ("gather_shape" or "cut_log2") and its value."""
        n = ctypes.c_int32()
        self._check("kde_autotune_table", self.lib.kde_autotune_table(self.h, 0, None, None, None,
                                                                      ctypes.addressof(n)))
        cap = n.value
        keys = np.zeros(max(cap, 1), dtype=np.uint64)
        kinds = np.zeros(max(cap, 1), dtype=np.int32)
        vals = np.zeros(max(cap, 1), dtype=np.float64)
        self._check("kde_autotune_table", self.lib.kde_autotune_table(self.h, cap, keys.ctypes.data, kinds.ctypes.data,
                                                                      vals.ctypes.data, ctypes.addressof(n)))
        out = []
        for k, t, v in zip(keys[:cap], kinds[:cap], vals[:cap]):
            k = int(k)
            out.append({"Ng": k & 0xFFFF, "log2_N": (k >> 16) & 0xFF, "width_class": (k >> 24) & 0xFF,
                        "kind": "gather_shape" if t == 0 else "cut_log2",
                        "value": int(v) if t == 0 else float(v)})
        return out

    def autotune_save(self, path):
        """Writes the autotuner's choices (autotune_table) to a JSON file."""
        with open(path, "w") as f:
            json.dump(self.autotune_table(), f, indent=1)

    def autotune_load(self, path):
        """kde_autotune_set from a JSON file written by autotune_save: the keys it lists are
        not tuned again."""
        with open(path) as f:
            tab = json.load(f)
        keys = np.array([e["Ng"] | (e["log2_N"] << 16) | (e["width_class"] << 24) for e in tab], dtype=np.uint64)
        kinds = np.array([0 if e["kind"] == "gather_shape" else 1 for e in tab], dtype=np.int32)
        vals = np.array([e["value"] for e in tab], dtype=np.float64)
        n = len(tab)
        self._check("kde_autotune_set", self.lib.kde_autotune_set(self.h, n, keys.ctypes.data if n else None,
                                                                  kinds.ctypes.data if n else None,
                                                                  vals.ctypes.data if n else None))

    def set_launch_overlap(self, on: bool = True):
        """kde_set_launch_overlap: programmatic dependent launches in the FP32 step chain."""
        self._check("kde_set_launch_overlap", self.lib.kde_set_launch_overlap(self.h, int(on)))

    def autotune_entries(self) -> int:
        """kde_autotune_entries: number of keys tuned so far."""
        n = ctypes.c_int32()
        self._check("kde_autotune_entries", self.lib.kde_autotune_entries(self.h, ctypes.addressof(n)))
        return n.value

    def profile_enable(self, on: bool = True):
        """kde_profile_enable: start (or stop) recording per-kernel device times."""
        self._check("kde_profile_enable", self.lib.kde_profile_enable(self.h, int(on)))

    def profile_read(self, kernel: str):
        """kde_profile_read: (total ms, launches) of one kernel since profile_enable;
        kernel='all' gives (0, number of all kernel launches)."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        kid = -1 if kernel == "all" else self.PROF[kernel]
        self._check("kde_profile_read", self.lib.kde_profile_read(self.h, kid, ctypes.addressof(ms),
                                                                  ctypes.addressof(n)))
        return ms.value, n.value

    def probe_exp2(self, iters: int):
        ms = ctypes.c_double()
        ops = ctypes.c_int64()
        self._check("kde_probe_exp2", self.lib.kde_probe_exp2(self.h, int(iters), ctypes.addressof(ms),
                                                              ctypes.addressof(ops)))
        return ms.value, ops.value

    def probe_fma(self, iters: int):
        ms = ctypes.c_double()
        ops = ctypes.c_int64()
        self._check("kde_probe_fma", self.lib.kde_probe_fma(self.h, int(iters), ctypes.addressof(ms),
                                                            ctypes.addressof(ops)))
        return ms.value, ops.value


def deposit_noalloc(u, Ng: int, L: float, kappa=None, kappa_uniform: float = 0.0, weight=None, out=None,
                    dtype=None, stream=None):
    """kde_deposit_noalloc: the deposit without a context or any device allocation by the
    library (its scratch is a fixed device array; `out` may be preallocated by the caller)."""
    torch = _torch()
    lib = load_library()
    dtype = dtype or (kappa.dtype if kappa is not None else torch.float32)
    if out is None:
        out = torch.empty(int(Ng), dtype=dtype, device=u.device)
    stream = stream or torch.cuda.current_stream(u.device)
    flags = F64 if out.dtype == torch.float64 else 0
    rc = lib.kde_deposit_noalloc(_P(stream.cuda_stream), _ptr(u), _ptr(kappa), float(kappa_uniform), _ptr(weight),
                                 u.numel(), int(Ng), float(L), _ptr(out), flags)
    if rc != 0:
        raise KdeError("kde_deposit_noalloc", rc, "invalid arguments or CUDA launch failure")
    return out


def damping_rate(energy, dt: float) -> float:
    """kde_damping_rate: half the slope of ln W through its first two maxima after t = 0."""
    lib = load_library()
    W = np.ascontiguousarray(energy, dtype=np.float64)
    g = ctypes.c_double()
    rc = lib.kde_damping_rate(W.ctypes.data, W.size, float(dt), ctypes.addressof(g))
    if rc != 0:
        raise KdeError("kde_damping_rate", rc, "fewer than two energy maxima")
    return g.value


class PicState:
    """Device state of one PIC run; tensors are owned here, the struct mirrors pic_state."""

    def __init__(self, u, v, L: float, Ng: int, dt: float, kappa=None, kappa_uniform: float = 0.0, ids=None,
                 qm: float = -1.0, charge: float = -1.0, background: float = 1.0, width_every: int = 0,
                 cand=None, alpha: float = 0.5, kappa_min: float = 0.0, kappa_max: float = 1e6,
                 max_steps: int = 0, fd: bool = False, backstep: bool = True, cv_spectral: bool = False,
                 cv_pairs: bool = False,
                 width_ad: bool = False, ad_threshold: float = 0.01, adjust_rate: float = 0.05,
                 shape_order: int = 0, shape_h: float = 0.0):
        torch = _torch()
        self.u, self.v, self.kappa, self.id = u, v, kappa, ids
        f64 = v.dtype == torch.float64
        self.kappa_norm = torch.empty_like(kappa) if kappa is not None else None
        self.cand = None if cand is None else np.ascontiguousarray(cand, dtype=np.float64)
        dev = u.device
        self.energy = torch.zeros(max(max_steps, 1), dtype=torch.float64, device=dev)
        self.kappa_star = torch.zeros(max(max_steps, 1), dtype=torch.float64, device=dev)
        self.ad_log_p = torch.zeros(max(max_steps, 1), dtype=torch.float64, device=dev)
        self.max_steps = max_steps
        c = _PicState()
        c.N = u.numel()
        c.Ng = int(Ng)
        c.L, c.dt, c.qm, c.charge, c.background = float(L), float(dt), float(qm), float(charge), float(background)
        c.kappa_uniform = float(kappa_uniform)
        c.width_every = int(width_every)
        c.n_cand = 0 if self.cand is None else self.cand.size
        c.alpha, c.kappa_min, c.kappa_max = float(alpha), float(kappa_min), float(kappa_max)
        c.step = 0
        c.flags = ((F64 if f64 else 0) | (POISSON_FD if fd else 0) | (0 if backstep else PIC_NO_BACKSTEP)
                   | (CV_SPECTRAL if cv_spectral else 0) | (CV_PAIRS if cv_pairs else 0))
        c.width_ad = int(bool(width_ad))
        c.ad_threshold, c.adjust_rate = float(ad_threshold), float(adjust_rate)
        c.ad_log_pth, c.h_target, c.n_opt = 0.0, 0.0, 0
        c.shape_order, c.shape_h = int(shape_order), float(shape_h)
        self.c = c

    def _sync_in(self):
        c = self.c
        c.u, c.v = _ptr(self.u), _ptr(self.v)
        c.kappa, c.kappa_norm, c.id = _ptr(self.kappa), _ptr(self.kappa_norm), _ptr(self.id)
        c.cand = None if self.cand is None else self.cand.ctypes.data
        ok = self.max_steps > 0
        c.energy = _ptr(self.energy) if ok else None
        c.kappa_star = _ptr(self.kappa_star) if ok else None
        c.ad_log_p = _ptr(self.ad_log_p) if ok else None

    @property
    def step(self) -> int:
        return self.c.step

    _ARRAYS = ("u", "v", "kappa", "kappa_norm", "id", "energy", "kappa_star", "ad_log_p")

    def snapshot(self):
        """Copies of the state's arrays (each on its own device) and of every scalar of the
        state; restore() puts them back, after which stepping repeats the run bit for bit."""
        arrs = {n: getattr(self, n).clone() for n in self._ARRAYS if getattr(self, n) is not None}
        scal = {f: getattr(self.c, f) for f, t in _PicState._fields_ if t is not _P}
        return arrs, scal

    def restore(self, snap):
        """Put back a snapshot() of this state (copies into the state's own tensors)."""
        arrs, scal = snap
        for n, t in arrs.items():
            getattr(self, n).copy_(t)
        for f, v in scal.items():
            setattr(self.c, f, v)

    def save(self, path):
        """Checkpoint the run to one .npz file: the particle arrays, the histories, the
        candidate list and every scalar of the state (step counter, widths, the width
        schedule's and the AD schedule's state).  Host-side copies only."""
        out = {}
        for name in self._ARRAYS:
            t = getattr(self, name)
            if t is not None:
                out["a_" + name] = t.detach().cpu().numpy()
        if self.cand is not None:
            out["cand"] = self.cand
        scal = {f: getattr(self.c, f) for f, t in _PicState._fields_ if t is not _P}
        out["scalars"] = np.array(json.dumps(scal))
        out["max_steps"] = np.array(self.max_steps)
        np.savez(path, **out)

    @classmethod
    def load(cls, path, device="cuda:0"):
        """The state saved by save(), on `device`; stepping it continues the saved run bit
        for bit."""
        torch = _torch()
        z = np.load(path, allow_pickle=False)
        a = {k[2:]: torch.from_numpy(z[k].copy()).to(device) for k in z.files if k.startswith("a_")}
        scal = json.loads(str(z["scalars"]))
        st = cls.__new__(cls)
        st.u, st.v = a["u"], a["v"]
        st.kappa, st.kappa_norm, st.id = a.get("kappa"), a.get("kappa_norm"), a.get("id")
        st.energy, st.kappa_star, st.ad_log_p = a["energy"], a["kappa_star"], a["ad_log_p"]
        st.cand = z["cand"] if "cand" in z.files else None
        st.max_steps = int(z["max_steps"])
        c = _PicState()
        for f, v in scal.items():
            setattr(c, f, v)
        st.c = c
        return st


class Ensemble:
    """kde_ensemble_*: R independent PIC realisations in concatenated device arrays.

    u (int32 view of the uint32 codes) and v (float32) are CUDA tensors of sum(N) entries,
    realisation r in N[r] consecutive slots; the ensemble keeps references to them."""

    def __init__(self, ctx: "Context", N, Ng, kappa, L: float, dt: float, u, v):
        self.ctx = ctx
        self.N = np.ascontiguousarray(N, dtype=np.int64)
        self.Ng = np.ascontiguousarray(Ng, dtype=np.int32)
        k = np.ascontiguousarray(kappa, dtype=np.float64)
        self.u, self.v = u, v
        h = _P()
        ctx._check("kde_ensemble_create", ctx.lib.kde_ensemble_create(
            ctx.h, ctypes.byref(h), self.N.size, self.N.ctypes.data, self.Ng.ctypes.data, k.ctypes.data,
            float(L), float(dt), _ptr(u), _ptr(v)))
        self.h = h

    @property
    def R(self):
        return self.N.size

    def set_widths(self, kappa):
        k = np.ascontiguousarray(kappa, dtype=np.float64)
        self.ctx._check("kde_ensemble_set_widths", self.ctx.lib.kde_ensemble_set_widths(self.h, k.ctypes.data))

    def set_shape(self, order: int, h: float = 0.0):
        """Standard PIC with the B-spline shape of degree `order` (0: back to the von Mises KDE)."""
        self.ctx._check("kde_ensemble_set_shape", self.ctx.lib.kde_ensemble_set_shape(self.h, int(order), float(h)))

    def mise(self, alpha: float, mode: int = 1):
        torch = _torch()
        out = torch.empty(self.R, dtype=torch.float64, device=self.u.device)
        self.ctx._check("kde_ensemble_mise", self.ctx.lib.kde_ensemble_mise(self.h, float(alpha), int(mode),
                                                                             _ptr(out)))
        return out

    def run(self, n_steps: int, energy=None, use_graph: bool = True):
        if energy is not None and energy.numel() < self.R * int(n_steps):
            raise KdeError("kde_ensemble_run", 1, "energy must hold R * n_steps values")
        self.ctx._check("kde_ensemble_run", self.ctx.lib.kde_ensemble_run(self.h, int(n_steps), _ptr(energy),
                                                                           int(use_graph)))

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.kde_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """kde_server_*: continuous-batching request server over host numpy buffers.

    submit() copies nothing on the host: it keeps references to the numpy arrays until
    wait() returns for the ticket (the library reads and writes them from its slots)."""

    def __init__(self, device: int = 0, n_slots: int = 4, hbm_budget_bytes: int = 100 << 30):
        self.lib = load_library()
        h = _P()
        rc = self.lib.kde_server_create(ctypes.byref(h), int(device), int(n_slots), int(hbm_budget_bytes))
        if rc != 0:
            raise KdeError("kde_server_create", rc, "cannot start the server")
        self.h = h
        self.keep = {}

    def submit(self, kind, u, L, Ng=1, kappa=None, kappa_uniform=0.0, v=None, field=None, cand=None, n_steps=0,
               dt=0.0, out=None, out64=None, flags=0):
        u = np.ascontiguousarray(u, dtype=np.uint32)
        arrs = [u]
        r = _Request()
        r.kind, r.N, r.Ng, r.L = int(kind), u.size, int(Ng), float(L)
        r.u = u.ctypes.data

        def f32(a):
            a = np.ascontiguousarray(a, dtype=np.float32)
            arrs.append(a)
            return a

        if kappa is not None:
            r.kappa = f32(kappa).ctypes.data
        r.kappa_uniform = float(kappa_uniform)
        if v is not None:
            r.v = f32(v).ctypes.data
        if field is not None:
            r.field = f32(field).ctypes.data
        if cand is not None:
            c = np.ascontiguousarray(cand, dtype=np.float64)
            arrs.append(c)
            r.cand, r.n_cand = c.ctypes.data, c.size
        r.n_steps, r.dt = int(n_steps), float(dt)
        am = np.zeros(1, dtype=np.int32)
        arrs.append(am)
        r.out_argmin = am.ctypes.data
        if out is not None:
            r.out = out.ctypes.data
            arrs.append(out)
        if out64 is not None:
            r.out64 = out64.ctypes.data
            arrs.append(out64)
        r.flags = int(flags)
        t = _I64()
        rc = self.lib.kde_server_submit(self.h, ctypes.byref(r), ctypes.byref(t))
        if rc != 0:
            raise KdeError("kde_server_submit", rc, "invalid request")
        self.keep[t.value] = (arrs, am)
        return t.value

    def wait(self, ticket, times=False):
        """kde_server_wait_times: (latency ms, service ms, argmin), plus the device-clock
        interval (start, end) in ms since the server started when times=True."""
        t = (ctypes.c_double * 4)()
        msg = ctypes.create_string_buffer(512)
        rc = self.lib.kde_server_wait_msg(self.h, int(ticket), ctypes.addressof(t), msg, 512)
        arrs, am = self.keep.pop(ticket)
        if rc != 0:
            raise KdeError("kde_server_wait", rc, msg.value.decode(errors="replace") or "request failed")
        if times:
            return t[0], t[1], int(am[0]), (t[2], t[3])
        return t[0], t[1], int(am[0])

    def cancel(self, ticket) -> int:
        """kde_server_cancel: 0 if the queued request was cancelled, else the status code."""
        return int(self.lib.kde_server_cancel(self.h, int(ticket)))

    def stats(self) -> dict:
        """kde_server_stats: HBM accounting and counters."""
        a = (ctypes.c_int64 * 8)()
        rc = self.lib.kde_server_stats(self.h, ctypes.addressof(a))
        if rc != 0:
            raise KdeError("kde_server_stats", rc, "bad server")
        keys = ["committed", "committed_peak", "budget", "served", "cancelled", "queued", "trims", "held"]
        return dict(zip(keys, list(a)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.kde_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
