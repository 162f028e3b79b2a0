"""The allocation-free deposit, kde_deposit_noalloc, called through the C ABI.

Callers that cannot allocate device memory while they run (work recorded into
CUDA graphs, hosts whose allocator policy forbids device allocations after
start-up, real-time loops) use this entry point instead of kde_deposit: it
takes a stream instead of a context and keeps its scratch in a fixed device
array inside the library.  Its output must match kde_deposit's within the
deposit tolerance of the other tests (1e-5 relative L2 in FP32, 1e-10 in
FP64), on two calls in a row (the shared scratch keeps the previous call's
contents), for sorted and unsorted particles; and it must match the FP64 oracle
within the same tolerances while the device's free memory stays the same across
calls.  This file is collected last so that a stop-at-first-failure run has
already run every other test.
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


def test_noalloc_matches_oracle_and_allocates_nothing(kp, oracle):
    # every buffer exists before the first call; after it (which may load the
    # module), repeated calls leave the device's free memory exactly where it was
    lib = kp.load_library()
    L = 4 * math.pi
    cases = [
        dict(N=30_011, Ng=256, kappa_u=120.0, f64=False),
        dict(N=6_000, Ng=333, per_particle=True, weights=True, f64=False),
        dict(N=3_000, Ng=64, kappa_u=25.0, f64=True),
    ]
    prepared = []
    for cs in cases:
        N, Ng, f64 = cs["N"], cs["Ng"], cs["f64"]
        u, _ = I.landau_load(N + 1, N, L, 0.05, 1.0)
        u = u[np.argsort(I.uniforms(N, 10, N))]
        dt = torch.float64 if f64 else torch.float32
        kap = I.log_uniform(N, I.STREAM_KAPPA, N, 5.0, 5e3) if cs.get("per_particle") else None
        w = 0.5 + I.uniforms(N, 8, N) if cs.get("weights") else None
        kap_d = None if kap is None else to_dev(kap, dt)
        w_d = None if w is None else to_dev(w, dt)
        # the oracle gets exactly the values the device holds
        kap_o = None if kap is None else kap_d.double().cpu().numpy()
        w_o = None if w is None else w_d.double().cpu().numpy()
        ref = oracle.deposit(I.from_fixed(u, L), Ng, L, kappa=kap_o, kappa_u=cs.get("kappa_u", 0.0), w=w_o)
        outs = [torch.full((Ng,), float("nan"), dtype=dt, device="cuda:0") for _ in range(3)]
        prepared.append((cs, to_dev_u(u), kap_d, w_d, ref, outs, 1e-10 if f64 else 1e-5))
    torch.cuda.synchronize()
    free0 = None
    for k in range(3):
        for cs, ud, kap_d, w_d, ref, outs, tol in prepared:
            rc = call(lib, ud, cs["Ng"], L, outs[k], kappa=kap_d, kappa_u=cs.get("kappa_u", 0.0), weight=w_d,
                      f64=cs["f64"])
            assert rc == 0
        torch.cuda.synchronize()
        free = torch.cuda.mem_get_info()[0]
        if k == 0:
            free0 = free
        else:
            assert free == free0, (free0, free)
    for cs, ud, kap_d, w_d, ref, outs, tol in prepared:
        for out in outs:
            assert rel_l2(out.cpu().numpy(), ref) <= tol, cs
