"""Speculative thresholds against the CPU oracle.

With the range computed (one field, stage 2 on), the stage kernel merges
each block's min / max into the header's keys itself and thresholds the
block at t_lo <= t, the threshold of the range known so far (the keys
merged so far and a subsample of every 4th row of every 4th z-plane);
stage 2 then drops the details below the exact t.  Streams must stay
byte-identical to the oracle's, which computes t first, also where t_lo
is far below t for most blocks (the range's extremes in one late voxel
the subsample misses), with NaN in the field, and with every value NaN.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import describe_diff, gpu_compress, gpu_decompress

pytestmark = pytest.mark.gpu

KINDS = (O.W4, O.W4LI, O.W3AI)


def _smooth(shape, dtype, seed):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64) for n in shape), indexing="ij")
    f = 3 * np.sin(x / 5.3 + rng.random()) * np.cos(y / 4.1) + np.sin(z / 2.9)
    return (f + 1e-3 * rng.standard_normal(shape)).astype(dtype)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("block,dtype,shape", [(32, np.float32, (96, 64, 128)), (16, np.float32, (48, 64, 80)),
                                                (8, np.float32, (32, 24, 40)), (16, np.float64, (48, 32, 64)),
                                                (8, np.float64, (24, 24, 32))])
def test_late_extreme_the_subsample_misses(kind, block, dtype, shape):
    """One voxel of the last block (row y = 1, plane z = last - 2: on no
    sampled row) holds the range: every earlier block keeps a superset."""
    f = _smooth(shape, dtype, seed=block + kind)
    f[-3, -(block - 1), -2] = 400.0
    for eps in (1e-3, 1e-5):
        want = O.compress(f, block, kind, eps)
        got = gpu_compress(f, block, kind, eps)
        assert got == want, describe_diff(got, want)
    np.testing.assert_array_equal(gpu_decompress(want).view(np.uint8), O.decompress(want).view(np.uint8))


@pytest.mark.parametrize("excess", (5e-4, 2e-3))
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("block,dtype,shape", [(32, np.float32, (96, 64, 128)), (16, np.float32, (48, 64, 80)),
                                                (8, np.float32, (32, 24, 40)), (16, np.float64, (48, 32, 64))])
def test_range_just_beyond_the_subsample(kind, block, dtype, shape, excess):
    """The field is clipped to its subsample's range (every 4th row of every
    4th z-plane), then one voxel on no sampled row exceeds it by `excess` of
    the range: t = (1 + excess) t_lo.  0.05 % lies within t_lo's near bound
    (1 + 2^-10): only the slots marked near are tested; 0.2 % lies beyond
    it: every slot is.  Small and large payloads (eps down to 1e-5)."""
    f = _smooth(shape, dtype, seed=3 * block + kind)
    s = f[::4, ::4, :]
    lo, hi = float(s.min()), float(s.max())
    f = np.clip(f, lo, hi).astype(dtype)
    f[-3, -(block - 1), -2] = hi + excess * (hi - lo)
    for eps in (1e-3, 1e-4, 1e-5):
        want = O.compress(f, block, kind, eps)
        got = gpu_compress(f, block, kind, eps)
        assert got == want, describe_diff(got, want)


@pytest.mark.parametrize("kind", KINDS)
def test_negative_extreme_first_then_positive_late(kind):
    f = _smooth((64, 64, 96), np.float32, seed=9)
    f[1, 1, 1] = -50.0      # in block 0, on no sampled row
    f[-2, -3, -5] = 75.0    # in the last block
    want = O.compress(f, 32, kind, 1e-3)
    got = gpu_compress(f, 32, kind, 1e-3)
    assert got == want, describe_diff(got, want)


def test_nan_values_with_stage2():
    """Header min / max / t equal the oracle's (NaN ignored by the range),
    decoded NaN positions and every other value equal."""
    f = _smooth((64, 32, 64), np.float32, seed=5)
    f[3, 4, 5] = np.nan
    f[40, 1, 30] = np.nan
    f[63, 31, 63] = np.nan
    got = gpu_compress(f, 32, O.W3AI, 1e-3)
    ref = O.compress(f, 32, O.W3AI, 1e-3)
    hg, hr = O.read_header(got), O.read_header(ref)
    assert hg["min"] == hr["min"] and hg["max"] == hr["max"] and hg["t"] == hr["t"]
    rec, want = gpu_decompress(got), O.decompress(ref)
    np.testing.assert_array_equal(np.isnan(rec), np.isnan(want))
    ok = ~np.isnan(want)
    np.testing.assert_array_equal(rec[ok].view(np.uint32), want[ok].view(np.uint32))


def test_every_value_nan():
    f = np.full((32, 32, 32), np.nan, np.float32)
    got = gpu_compress(f, 32, O.W3AI, 1e-3)
    ref = O.compress(f, 32, O.W3AI, 1e-3)
    hg, hr = O.read_header(got), O.read_header(ref)
    for key in ("min", "max", "t", "range"):
        assert (hg[key] == hr[key]) or (np.isnan(hg[key]) and np.isnan(hr[key])), key
    assert np.isnan(gpu_decompress(got)).all()
