"""Parity at full size, in the benchmark's launch configuration.

The 1024^3 FP32 pressure field (32^3 blocks, W3ai, eps = 1e-3 * range,
stage 2 on) and the 768^3 FP64 density field (16^3 blocks, and 32^3 blocks
for the slab kernels) are compressed
and decompressed on the GPU through the C ABI exactly as bench.py does; the
oracle then re-encodes a seeded sample of blocks one by one with the
threshold it derives from its own min/max of the whole field.  Header
fields, the sampled chunks (byte for byte) and the sampled decoded blocks
(bit for bit) must agree; every chunk's offset must be consistent.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


def _check(f, B, kind, eps, nsample, seed):
    import torch
    from paper_1903_07761_gb300 import cz
    t = torch.from_numpy(f).cuda()
    out, nb = cz.compress(t, block=B, kind=kind, eps=eps)
    rec = cz.decompress(out, nbytes=int(nb.item()))
    torch.cuda.synchronize()
    n = int(nb.item())
    stream = out[:n].cpu().numpy().tobytes()
    del out
    h = O.read_header(stream)
    mn, mx = O.minmax(f)
    rng_ = (mx - mn) if mn <= mx else 0.0
    tt = np.dtype(f.dtype).type(O.threshold(eps, O.EPS_REL, rng_))
    assert h["min"] == mn and h["max"] == mx and h["range"] == rng_
    assert h["t"] == float(tt)
    d0, offs = O.chunk_table(stream)
    nz, ny, nx = f.shape
    nbx, nby, nbz = nx // B, ny // B, nz // B
    assert len(offs) == nbx * nby * nbz + 1 and offs[-1] == n - d0 and np.all(np.diff(offs) >= 8)
    rs = np.random.default_rng(seed)
    sample = set(rs.choice(len(offs) - 1, nsample, replace=False).tolist()) | {0, len(offs) - 2}
    for b in sorted(sample):
        bx, by, bz = b % nbx, (b // nbx) % nby, b // (nbx * nby)
        blk = f[bz * B:(bz + 1) * B, by * B:(by + 1) * B, bx * B:(bx + 1) * B]
        want = O.encode_block(kind, float(tt), blk, True)
        got = stream[d0 + offs[b]: d0 + offs[b + 1]]
        assert got == want, f"block {b}"
        dec = O.decode_block(kind, B, f.dtype, want, True)
        r = rec[bz * B:(bz + 1) * B, by * B:(by + 1) * B, bx * B:(bx + 1) * B].cpu().numpy()
        np.testing.assert_array_equal(r.view(np.uint8), dec.view(np.uint8))


def test_1024_cubed_fp32_pressure_field():
    from paper_1903_07761_gb300 import inputs
    f = inputs.cavitation("p", 1024, np.float32, seed=2000)
    _check(f, 32, O.W3AI, 1e-3, nsample=96, seed=1)


@pytest.mark.parametrize("B", [16, 32])
def test_768_cubed_fp64_density_field(B):
    from paper_1903_07761_gb300 import inputs
    f = inputs.cavitation("rho", 768, np.float64, seed=2001)
    _check(f, B, O.W3AI, 1e-3, nsample=96 if B == 16 else 48, seed=2)
