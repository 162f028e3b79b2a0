"""The allocation-free deposit, kde_deposit_noalloc, called through the C ABI.

Callers that cannot allocate device memory while they run (work recorded into
CUDA graphs, hosts whose allocator policy forbids device allocations after
start-up, real-time loops) use this entry point instead of kde_deposit: it
takes a stream instead of a context and keeps its scratch in a fixed device
array inside the library.  Its output must match kde_deposit's within the
deposit tolerance of the other tests (1e-5 relative L2 in FP32, 1e-10 in
FP64), on two calls in a row (the shared scratch keeps the previous call's
contents), for sorted and unsorted particles.  This file is collected last so
that a stop-at-first-failure run has already run every other test.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import kde_inputs as I
from conftest import rel_l2, to_dev, to_dev_u

pytestmark = pytest.mark.gpu


def call(lib, u, Ng, L, out, kappa=None, kappa_u=0.0, weight=None, f64=False):
    stream = torch.cuda.current_stream().cuda_stream
    p = lambda t: None if t is None else t.data_ptr()
    return lib.kde_deposit_noalloc(ctypes.c_void_p(stream), p(u), p(kappa), float(kappa_u), p(weight), u.numel(),
                                   int(Ng), float(L), p(out), 1 if f64 else 0)


@pytest.mark.parametrize("order", ["as generated", "shuffled"])
def test_noalloc_matches_deposit_twice(ctx, kp, order):
    lib = kp.load_library()
    L = 4 * math.pi
    cases = [
        dict(N=70_001, Ng=256, kappa_u=400.0),
        dict(N=5_000, Ng=100, per_particle=True, weights=True),
        dict(N=4_096, Ng=64, kappa_u=30.0, f64=True),
        dict(N=20_000, Ng=4096, kappa_u=2e4),
    ]
    for cs in cases:
        N, Ng = cs["N"], cs["Ng"]
        u, _ = I.landau_load(N, N, L, 0.05, 1.0)
        if order == "shuffled":
            u = u[np.argsort(I.uniforms(N, 9, N))]
        f64 = cs.get("f64", False)
        dt = torch.float64 if f64 else torch.float32
        ud = to_dev_u(u)
        kap = to_dev(I.log_uniform(N, I.STREAM_KAPPA, N, 5.0, 5e3), dt) if cs.get("per_particle") else None
        w = to_dev(0.5 + I.uniforms(N, 8, N), dt) if cs.get("weights") else None
        ref = ctx.deposit(ud, Ng, L, kappa=kap, kappa_uniform=cs.get("kappa_u", 0.0), weight=w, dtype=dt)
        ctx.sync()
        tol = 1e-10 if f64 else 1e-5
        for _ in range(2):
            out = torch.full((Ng,), float("nan"), dtype=dt, device="cuda:0")
            rc = call(lib, ud, Ng, L, out, kappa=kap, kappa_u=cs.get("kappa_u", 0.0), weight=w, f64=f64)
            assert rc == 0
            torch.cuda.synchronize()
            assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) <= tol


def test_noalloc_rejects_oversized_grid_and_bad_arguments(kp):
    lib = kp.load_library()
    u = to_dev_u(np.arange(100, dtype=np.uint32) * 4000)
    out = torch.empty(8192, device="cuda:0")
    assert call(lib, u, 4097, 1.0, out, kappa_u=5.0) == 1   # beyond the 4096-node maximum
    assert call(lib, u, 64, 1.0, out, kappa_u=0.0) == 1     # no width given
    assert call(lib, u, 64, -1.0, out, kappa_u=5.0) == 1    # bad domain
    assert call(lib, u[:0], 64, 1.0, out, kappa_u=5.0) == 0  # empty input gives zeros
    torch.cuda.synchronize()
    assert torch.all(out[:64] == 0)
