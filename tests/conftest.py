import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running parity case at full configuration size")


@pytest.fixture(scope="session")
def oracle():
    import oracle as O
    O.build()
    return O


@pytest.fixture(scope="session")
def kp():
    """The CUDA binding; builds libkdepic first (nvcc)."""
    import __graft_entry__
    __graft_entry__.build()
    import paper_1804_11174_gb300 as kp
    return kp


@pytest.fixture(scope="session")
def ctx(kp):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = kp.Context(0)
    yield c
    c.close()


def to_dev_u(u_np):
    """uint32 position codes -> int32 CUDA tensor with the same bits."""
    import numpy as np
    import torch
    return torch.from_numpy(np.ascontiguousarray(u_np, dtype=np.uint32).view(np.int32)).to("cuda:0")


def to_dev(a, dtype=None):
    import numpy as np
    import torch
    dtype = dtype or torch.float32
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda:0", dtype=dtype)


def rel_l2(a, b):
    import numpy as np
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
