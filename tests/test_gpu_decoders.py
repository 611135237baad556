"""Both block decoders against the CPU oracle.

Two decoders, chosen with a test hook (czi_set_decoder): one CTA per block
(mode 0, the default) and, for FP32 blocks of edge 16 and 32, two CTAs per
block (mode 1; one per z-half, each rebuilding the coarse cube and its
z-step halo from the payload).  Both must give fields bit-identical to
the oracle's: every kind, stage 2 on and off, ragged block grids with
several blocks per CTA, eps = 0 (payloads above the decoders' shared-memory
buffers, whose values are read from global memory), random access and
corrupt chunks.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from gpu_helpers import gpu_compress, gpu_decompress

pytestmark = pytest.mark.gpu

KINDS = (O.W4, O.W4LI, O.W3AI)


@pytest.fixture(params=[0, 1], ids=["whole", "half"])
def decoder(request):
    from paper_1903_07761_gb300 import cz
    L = cz.lib()
    L.czi_set_decoder.argtypes = [C.c_int]
    L.czi_set_decoder.restype = C.c_int
    assert L.czi_set_decoder(request.param) == cz.OK
    yield request.param
    assert L.czi_set_decoder(0) == cz.OK


def _field(shape, dtype, seed, noise=1e-3):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64) for n in shape), indexing="ij")
    f = 40 + 15 * np.sin(x / 5.3 + rng.random()) * np.cos(y / 4.1) + 4 * np.sin(z / 2.9)
    f += 6 * np.exp(-((x - shape[2] / 3) ** 2 + (z - shape[0] / 2) ** 2) / 20.0)
    f += noise * rng.standard_normal(shape)
    return f.astype(dtype)


@pytest.mark.parametrize("stage2", [True, False])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("block,shape", [(32, (64, 96, 160)), (16, (48, 32, 80))])
def test_decoded_field_bit_identical(decoder, block, shape, kind, stage2):
    f = _field(shape, np.float32, seed=block * 3 + kind)
    for eps in (1e-2, 1e-3, 1e-5):
        s = O.compress(f, block, kind, eps, stage2=stage2)
        rec = gpu_decompress(s)
        np.testing.assert_array_equal(rec.view(np.uint32), O.decompress(s).view(np.uint32))


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("block", [32, 16])
def test_every_detail_kept(decoder, block, kind):
    """eps = 0 on noise: every coefficient is stored; the 32^3 payloads
    (132 KiB) exceed the decoders' buffers, so values come from global memory."""
    rng = np.random.default_rng(block + kind)
    f = rng.standard_normal((block, 2 * block, 3 * block)).astype(np.float32)
    for stage2 in (True, False):
        s = O.compress(f, block, kind, 0.0, stage2=stage2)
        rec = gpu_decompress(s)
        np.testing.assert_array_equal(rec.view(np.uint32), O.decompress(s).view(np.uint32))


def test_many_blocks_per_cta(decoder):
    """A grid of 2048 blocks: every CTA of the persistent decoders takes
    several blocks (carries across the block grid's x and y)."""
    f = _field((256, 256, 256), np.float32, seed=7)
    s = gpu_compress(f, 32, O.W3AI, 1e-3)
    rec = gpu_decompress(s)
    want = O.decompress(s)
    np.testing.assert_array_equal(rec.view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("kind", KINDS)
def test_random_access_tiles(decoder, kind):
    import torch
    from paper_1903_07761_gb300 import cz
    f = _field((64, 64, 96), np.float32, seed=kind)
    s = O.compress(f, 32, kind, 1e-3)
    want = O.decompress(s)
    st = torch.from_numpy(np.frombuffer(s, np.uint8).copy()).cuda()
    ids = [11, 0, 5, 5, 3]  # x-fastest over a 3 x 2 x 2 block grid
    tiles = cz.decompress_blocks(st, torch.tensor(ids, dtype=torch.int32, device="cuda"), nbytes=len(s)).cpu().numpy()
    for t, b in zip(tiles, ids):
        bx, by, bz = b % 3, (b // 3) % 2, b // 6
        np.testing.assert_array_equal(t.view(np.uint32),
                                      want[bz * 32:(bz + 1) * 32, by * 32:(by + 1) * 32,
                                           bx * 32:(bx + 1) * 32].view(np.uint32))


def test_corrupt_chunk_gives_zeros_and_status(decoder):
    import torch
    from paper_1903_07761_gb300 import cz
    f = _field((32, 32, 64), np.float32, seed=3)
    s = bytearray(O.compress(f, 32, O.W3AI, 1e-3, stage2=False))
    data0, offs = O.chunk_table(bytes(s))
    # block 1's nnz no longer matches its mask
    o = data0 + int(offs[1])
    s[o:o + 4] = (int.from_bytes(s[o:o + 4], "little") + 1).to_bytes(4, "little")
    st = torch.from_numpy(np.frombuffer(bytes(s), np.uint8).copy()).cuda()
    with pytest.raises(cz.CzError) as e:
        cz.decompress(st, nbytes=len(s))
    assert e.value.code == cz.ERR_CORRUPT
    ws = cz.Workspace()
    out = cz.decompress(st, nbytes=len(s), ws=ws, check=False).cpu().numpy()
    want = O.decompress(O.compress(f, 32, O.W3AI, 1e-3, stage2=False))
    np.testing.assert_array_equal(out[:, :, :32].view(np.uint32), want[:, :, :32].view(np.uint32))
    assert not out[:, :, 32:].any()
