"""GPU parity of the position encoding kde_pack_positions (periodic fixed point,
Sec. III.A periodic boundary) with the host encoding kde_inputs.to_fixed that
every oracle comparison is fed: integer codes, so the bar is bit-exact."""
import math

import numpy as np
import pytest
import torch

import kde_inputs as I

pytestmark = pytest.mark.gpu


def pack(ctx, x, L):
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to("cuda:0")
    u = ctx.pack_positions(xd, L)
    ctx.sync()
    return u.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("L", [4 * math.pi, 1.0, 3.0, 2.0 ** -7, 1e5])
def test_pack_positions_bit_exact(ctx, L):
    n = 300007                                         # ragged: not a multiple of the block
    inside = I.uniforms(31, 0, n) * L                  # [0, L)
    neg = -I.uniforms(31, 1, 1001) * 7.5 * L           # negative positions wrap
    big = L + I.uniforms(31, 2, 1001) * 1e6 * L        # positions >= L wrap
    last = L * (1.0 - 2.0 ** -33)                      # the last code below L
    specials = np.array([0.0, -0.0, L, -L, 2 * L, last, np.nextafter(L, 0.0), np.nextafter(0.0, 1.0),
                         -1e-300, -np.nextafter(0.0, 1.0), L * 0.5, L * (1.0 - 2.0 ** -32),
                         L * 2.0 ** -32, L * (2.0 ** -32 - 2.0 ** -60), 3.5 * L, -0.5 * L])
    x = np.concatenate([inside, neg, big, specials])
    got = pack(ctx, x, L)
    ref = I.to_fixed(x, L)
    assert got.dtype == np.uint32 and got.shape == ref.shape
    bad = np.nonzero(got != ref)[0]
    assert bad.size == 0, "first mismatches: %s" % [(float(x[i]), int(got[i]), int(ref[i])) for i in bad[:5]]
    s = got[-specials.size:]
    assert s[0] == 0 and s[2] == 0 and s[5] == 2 ** 32 - 1 and s[6] == 2 ** 32 - 1


def test_pack_positions_round_trip_of_codes(ctx):
    # x = u L / 2^32 rounded to FP64 (the oracle's positions): packing it gives the
    # host encoding bit for bit, and u itself or, where the product rounded down,
    # the code below it
    L = 4 * math.pi
    u, _ = I.landau_load(3, 1 << 16, L)
    u = np.concatenate([u, np.array([0, 1, 2 ** 31, 2 ** 32 - 2, 2 ** 32 - 1], dtype=np.uint32)])
    x = I.from_fixed(u, L)
    got = pack(ctx, x, L)
    assert np.array_equal(got, I.to_fixed(x, L))
    d = (u.astype(np.int64) - got.astype(np.int64)) % (1 << 32)
    assert np.all((d == 0) | (d == 1))
    # with L a power of two the product is exact and the codes come back unchanged
    got2 = pack(ctx, I.from_fixed(u, 2.0), 2.0)
    assert np.array_equal(got2, u)


def test_pack_positions_empty_and_bad_arguments(ctx, kp):
    e = torch.empty(0, dtype=torch.float64, device="cuda:0")
    assert ctx.pack_positions(e, 1.0).numel() == 0
    x = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    with pytest.raises(kp.KdeError):
        ctx.pack_positions(x, 0.0)
    with pytest.raises(kp.KdeError):
        ctx.pack_positions(x, -2.0)
