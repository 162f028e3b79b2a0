"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/kdepic.h declares."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "kdepic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("kde_", "pic_"))))


def test_header_declares_the_hot_path():
    names = declared_symbols()
    for n in ["kde_deposit", "kde_gather", "kde_cv", "pic_step", "kde_poisson", "kde_adapt_widths"]:
        assert n in names


def test_library_exports_every_declared_symbol(kp):
    lib = kp.load_library()
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_refuses_missing_library(kp, tmp_path):
    import pytest
    with pytest.raises(ImportError):
        kp.load_library(str(tmp_path / "nope.so"))


def test_damping_rate_host_entry(kp):
    import math
    import numpy as np
    t = 0.1 * np.arange(200)
    W = np.exp(-0.3 * t) * np.cos(1.4 * t + 0.3) ** 2 + 1e-12
    g = kp.damping_rate(W, 0.1)
    assert abs(g + 0.15) < 0.01


def test_null_context_is_rejected_on_the_host(kp):
    # argument checks run on the host before anything touches CUDA: a null context gives
    # KDE_EINVAL (1) and a readable error, with no GPU present
    import ctypes
    lib = kp.load_library()
    n = ctypes.c_int32(-1)
    assert lib.kde_set_autotune(None, 1) == 1
    assert lib.kde_autotune_entries(None, ctypes.addressof(n)) == 1 and n.value == -1
    assert lib.kde_autotune_table(None, 0, None, None, None, ctypes.addressof(n)) == 1 and n.value == -1
    assert lib.kde_set_truncation(None, ctypes.c_double(20.0)) == 1
    assert lib.kde_autotune_set(None, 0, None, None, None) == 1
    assert lib.kde_set_launch_overlap(None, 1) == 1
    assert lib.kde_sync(None) == 1
    assert lib.kde_destroy(None) == 1
    assert lib.kde_set_stream(None, None) == 1
    assert lib.kde_last_error(None) == b"null context"


def test_pic_state_snapshot_restore_on_host(kp, tmp_path):
    # the state's own copy helpers (no library call): a restored snapshot and a reloaded
    # checkpoint give back every array and every scalar of the state
    import numpy as np
    import torch
    N = 64
    st = kp.PicState(torch.arange(N, dtype=torch.int32), torch.linspace(-1, 1, N), 4.0, 16, 0.1,
                     kappa=torch.full((N,), 3.0), ids=torch.arange(N, dtype=torch.int32), width_every=5,
                     cand=np.array([1.0, 10.0]), max_steps=8)
    snap = st.snapshot()
    st.u += 7
    st.v.mul_(2)
    st.kappa.fill_(9.0)
    st.energy[3] = 1.5
    st.c.step, st.c.n_opt, st.c.h_target = 6, 2, 0.25
    st.save(tmp_path / "s.npz")
    st.restore(snap)
    assert st.c.step == 0 and st.c.n_opt == 0 and st.c.h_target == 0.0
    assert torch.equal(st.u, torch.arange(N, dtype=torch.int32)) and torch.equal(st.v, torch.linspace(-1, 1, N))
    assert torch.all(st.kappa == 3.0) and torch.all(st.energy == 0)
    back = kp.PicState.load(tmp_path / "s.npz", device="cpu")
    assert back.c.step == 6 and back.c.n_opt == 2 and back.c.h_target == 0.25
    assert torch.equal(back.u, torch.arange(N, dtype=torch.int32) + 7) and float(back.energy[3]) == 1.5
    assert back.c.width_every == 5 and back.c.Ng == 16 and back.c.N == N
