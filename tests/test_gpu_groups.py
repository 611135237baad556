"""Aggregate chunks on the GPU against the CPU oracle (Sec. 3, Exp. 2 and 3:
G consecutive blocks share one stage-2 chunk).

Streams must be byte-identical to the oracle's and decoded fields
bit-identical, for every kind, FP32 and FP64, every block edge and group
size the library takes, ragged block grids (a partial last group), groups
small enough for the shared-memory coder and, at eps = 0, groups that take
the large-group coder and decoder (payloads above 192 KiB); random access
decodes a block's whole group; a corrupt group chunk zeroes that group and
reports CZ_ERR_CORRUPT.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from gpu_helpers import describe_diff, gpu_compress, gpu_decompress

pytestmark = pytest.mark.gpu

KINDS = (O.W4, O.W4LI, O.W3AI)


def _field(shape, dtype, seed, noise=1e-3):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64) for n in shape), indexing="ij")
    f = 40 + 15 * np.sin(x / 5.3 + rng.random()) * np.cos(y / 4.1) + 4 * np.sin(z / 2.9)
    f += 6 * np.exp(-((x - shape[2] / 3) ** 2 + (z - shape[0] / 2) ** 2) / 20.0)
    f += noise * rng.standard_normal(shape)
    return f.astype(dtype)


# (block, dtype, group, shape): ragged grids (block counts not multiples of G)
CASES = [
    (32, np.float32, 4, (64, 96, 160)),    # 30 blocks
    (32, np.float32, 8, (64, 96, 160)),
    (16, np.float32, 16, (48, 80, 64)),    # 60 blocks
    (16, np.float64, 8, (48, 80, 64)),
    (8, np.float32, 16, (24, 40, 56)),     # 105 blocks
    (8, np.float64, 4, (24, 40, 56)),
    (32, np.float64, 4, (64, 64, 96)),     # 12 blocks: slab lane
]


@pytest.mark.parametrize("block,dtype,group,shape", CASES)
@pytest.mark.parametrize("kind", KINDS)
def test_group_streams_equal_the_oracle(block, dtype, group, shape, kind):
    f = _field(shape, dtype, seed=block * 7 + group + kind)
    for eps in (1e-2, 1e-4):
        want = O.compress(f, block, kind, eps, group=group)
        got = gpu_compress(f, block, kind, eps, group=group)
        assert got == want, describe_diff(got, want)
        rec = gpu_decompress(want)
        np.testing.assert_array_equal(rec.view(np.uint8), O.decompress(want).view(np.uint8))


@pytest.mark.parametrize("block,dtype,group,shape", [(32, np.float32, 8, (32, 64, 160)),
                                                     (16, np.float32, 16, (16, 48, 96)),
                                                     (32, np.float64, 4, (32, 32, 96)),
                                                     (16, np.float32, 4, (16, 48, 96))])
def test_large_groups_every_detail_kept(block, dtype, group, shape):
    """eps = 0 on noise: every coefficient is stored, so the group payloads
    (up to 1 MiB) exceed the shared-memory coder and take the large-group
    kernels (literal runs above 65535 words are split); 16^3 FP32 groups of
    4 (68 KiB) stay in shared memory."""
    rng = np.random.default_rng(block + group)
    f = rng.standard_normal(shape).astype(dtype)
    for kind in (O.W4, O.W3AI):
        want = O.compress(f, block, kind, 0.0, group=group)
        got = gpu_compress(f, block, kind, 0.0, group=group)
        assert got == want, describe_diff(got, want)
        rec = gpu_decompress(want)
        np.testing.assert_array_equal(rec.view(np.uint8), O.decompress(want).view(np.uint8))


def test_mixed_small_and_large_groups_with_zeroing():
    """Half of the field is noise at a tiny threshold (large groups), half
    smooth (small groups); Z8 bit zeroing on top."""
    f = _field((32, 64, 256), np.float32, seed=4)
    f[:, :, 128:] = np.random.default_rng(9).standard_normal((32, 64, 128)).astype(np.float32)
    for group in (4, 8):
        want = O.compress(f, 32, O.W3AI, 1e-7, group=group, zbits=8)
        got = gpu_compress(f, 32, O.W3AI, 1e-7, group=group, zbits=8)
        assert got == want, describe_diff(got, want)
        np.testing.assert_array_equal(gpu_decompress(want).view(np.uint8), O.decompress(want).view(np.uint8))


@pytest.mark.parametrize("decoder", [0, 1], ids=["whole", "half"])
def test_group_random_access(decoder):
    import torch
    from paper_1903_07761_gb300 import cz
    L = cz.lib()
    L.czi_set_decoder.argtypes = [C.c_int]
    L.czi_set_decoder.restype = C.c_int
    assert L.czi_set_decoder(decoder) == cz.OK
    try:
        f = _field((64, 64, 160), np.float32, seed=5)  # 5 x 2 x 2 = 20 blocks, groups of 8: 8, 8, 4
        for eps in (1e-3, 0.0):
            s = O.compress(f, 32, O.W4LI, eps, group=8)
            want = O.decompress(s)
            st = torch.from_numpy(np.frombuffer(s, np.uint8).copy()).cuda()
            ids = [19, 0, 7, 8, 8, 16, 3]
            tiles = cz.decompress_blocks(st, torch.tensor(ids, dtype=torch.int32, device="cuda"),
                                         nbytes=len(s)).cpu().numpy()
            for t, b in zip(tiles, ids):
                bx, by, bz = b % 5, (b // 5) % 2, b // 10
                np.testing.assert_array_equal(
                    t.view(np.uint32),
                    want[bz * 32:(bz + 1) * 32, by * 32:(by + 1) * 32, bx * 32:(bx + 1) * 32].view(np.uint32))
    finally:
        assert L.czi_set_decoder(0) == cz.OK


def test_corrupt_group_chunk_zeroes_its_group():
    import torch
    from paper_1903_07761_gb300 import cz
    f = _field((32, 32, 256), np.float32, seed=6)  # 8 blocks in x, groups of 4
    s = bytearray(O.compress(f, 32, O.W3AI, 1e-3, group=4))
    data0, offs = O.chunk_table(bytes(s))
    o = data0 + int(offs[1])  # group 1 (blocks 4..7): nnz of its first block beyond a block's details
    s[o:o + 4] = (32 ** 3).to_bytes(4, "little")
    st = torch.from_numpy(np.frombuffer(bytes(s), np.uint8).copy()).cuda()
    with pytest.raises(cz.CzError) as e:
        cz.decompress(st, nbytes=len(s))
    assert e.value.code == cz.ERR_CORRUPT
    out = cz.decompress(st, nbytes=len(s), ws=cz.Workspace(), check=False).cpu().numpy()
    want = O.decompress(O.compress(f, 32, O.W3AI, 1e-3, group=4))
    np.testing.assert_array_equal(out[:, :, :128].view(np.uint32), want[:, :, :128].view(np.uint32))
    assert not out[:, :, 128:].any()


def test_server_refuses_group_compression_and_decodes_group_streams():
    import torch
    from paper_1903_07761_gb300 import cz
    f = _field((32, 64, 96), np.float32, seed=11)
    want_stream = O.compress(f, 16, O.W3AI, 1e-3, group=8)
    st = torch.from_numpy(np.frombuffer(want_stream, np.uint8).copy()).cuda()
    ft = torch.from_numpy(f).cuda()
    out = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    rec = torch.zeros_like(ft)
    with cz.Server(1 << 28, 2) as srv:
        p = cz.params_for(f.shape, False, 16, "w3ai", 1e-3, group=8)
        with pytest.raises(cz.CzError) as e:
            srv.submit_compress(p, ft.data_ptr(), out.data_ptr(), out.numel(), 0)
        assert e.value.code == cz.ERR_ARG
        t = srv.submit_decompress(st.data_ptr(), len(want_stream), want_stream[:cz.HEADER_BYTES], rec.data_ptr(),
                                  rec.numel() * 4)
        res, _ = srv.wait(t)
        assert res == cz.OK
    np.testing.assert_array_equal(rec.cpu().numpy().view(np.uint32), O.decompress(want_stream).view(np.uint32))


def test_noalloc_takes_groups():
    import torch
    from paper_1903_07761_gb300 import cz
    f = _field((64, 64, 96), np.float32, seed=8)
    want = O.compress(f, 16, O.W4, 1e-3, group=16)
    p = cz.params_for(f.shape, False, 16, "w4", 1e-3, group=16)
    ft = torch.from_numpy(f).cuda()
    cap = cz.cz_compress_bound(p)
    out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert cz.cz_compress_noalloc(p, ft.data_ptr(), out.data_ptr(), cap, nb.data_ptr(), s) == cz.OK
    assert cz.cz_noalloc_status(s) == cz.OK
    torch.cuda.synchronize()
    got = out[:int(nb.item())].cpu().numpy().tobytes()
    assert got == want, describe_diff(got, want)


@pytest.mark.parametrize("block,f64,group", [(32, False, 4), (32, False, 8), (16, False, 16), (16, True, 8),
                                             (8, False, 16), (32, True, 4)])
def test_workspace_size_covers_group_decompression(block, f64, group):
    import ctypes as C
    from paper_1903_07761_gb300 import cz
    for shape in ((block, block, 30 * block), (4 * block, 4 * block, 4 * block)):
        p = cz.params_for(shape, f64, block, "w3ai", 1e-3, group=group)
        nb = (shape[0] // block) * (shape[1] // block) * (shape[2] // block)
        need = C.c_size_t()
        assert cz.lib().cz_decompress_blocks_workspace_size(C.byref(p), nb, C.byref(need)) == cz.OK
        assert cz.cz_workspace_size(p) >= need.value
