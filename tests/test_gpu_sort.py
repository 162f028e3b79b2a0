"""The stable counting sort by cell that every PIC step starts with (A1), seen through
pic_step with the push switched off (v = 0, no kick): the state comes back in the order of
a stable sort of the input by cell, with every payload moved alongside.  Sizes cover
ragged tails, several blocks per cell, a count table of more than one scan tile, the
largest grid, and the unit doubling that keeps the count table within its limit
(N = 2^22 at Ng = 4096).
"""
import math

import numpy as np
import pytest
import torch

import kde_inputs as I
from conftest import to_dev, to_dev_u

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,Ng", [(1, 64), (2047, 64), (100003, 100), ((1 << 20) + 123, 4096), (1 << 22, 4096),
                                  (4183125, 3072), (3000001, 2900)])
@pytest.mark.parametrize("steps", [1, 2])
def test_sort_is_stable_and_moves_payloads(ctx, kp, N, Ng, steps):
    # steps = 2: the second step's sort uses the counts that the first step's gather + push
    # added (the positions do not move, so the state must come back unchanged).  Ng near
    # 3072 with N ~ 2^22 needs longer units to fit the scatter's shared memory.
    L = 4 * math.pi
    u = I.to_fixed(I.random_positions(N % 977 + Ng, N, L, 0.05), L)
    kap = (5.0 + (np.arange(N) % 1000)).astype(np.float32)
    st = kp.PicState(to_dev_u(u), torch.zeros(N, device="cuda:0"), L, Ng, 0.1, kappa=to_dev(kap),
                     ids=torch.arange(N, dtype=torch.int32, device="cuda:0"), qm=0.0, max_steps=steps)
    ctx.pic_step(st, steps)
    ctx.sync()
    cell = (u.astype(np.uint64) * np.uint64(Ng)) >> np.uint64(32)
    order = np.argsort(cell, kind="stable")
    ids = st.id.cpu().numpy().view(np.uint32).astype(np.int64)
    np.testing.assert_array_equal(ids, order)
    np.testing.assert_array_equal(st.u.cpu().numpy().view(np.uint32), u[order])
    np.testing.assert_array_equal(st.kappa.cpu().numpy(), kap[order])
    assert np.all(st.v.cpu().numpy() == 0.0)
