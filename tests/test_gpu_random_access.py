"""Random access: decoding chosen blocks of a stream (cz_decompress_blocks)
gives exactly the oracle's decoded field, cut into those blocks."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


def _field(shape, dtype, seed):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64) for n in shape), indexing="ij")
    f = 40 + 15 * np.sin(x / 6.1 + rng.random()) * np.cos(y / 4.3) + 2 * np.sin(z / 2.9)
    f += 1e-3 * rng.standard_normal(shape)
    return f.astype(dtype)


def _blocks(field, B):
    nz, ny, nx = (n // B for n in field.shape)
    return field.reshape(nz, B, ny, B, nx, B).transpose(0, 2, 4, 1, 3, 5).reshape(-1, B, B, B)


@pytest.mark.parametrize("stage2", [True, False])
@pytest.mark.parametrize("kind", [O.W4, O.W4LI, O.W3AI])
@pytest.mark.parametrize("dtype,block,shape", [
    (np.float32, 32, (64, 96, 160)),
    (np.float64, 16, (32, 48, 64)),
    (np.float32, 8, (16, 24, 40)),
    (np.float64, 32, (32, 64, 96)),
    (np.float32, 64, (64, 64, 128)),
])
def test_decoded_blocks_equal_the_oracle_field_blocks(dtype, block, shape, kind, stage2):
    import torch
    from paper_1903_07761_gb300 import cz
    f = _field(shape, dtype, seed=block + kind)
    ref = O.compress(f, block, kind, 1e-3, stage2=stage2)
    want = _blocks(O.decompress(ref), block)
    nb = want.shape[0]
    rng = np.random.default_rng(7)
    ids = np.concatenate([[0, nb - 1], rng.integers(0, nb, 2 * nb), [nb - 1, 0]]).astype(np.int32)
    st = torch.from_numpy(np.frombuffer(ref, np.uint8).copy()).cuda()
    tiles = cz.decompress_blocks(st, torch.from_numpy(ids).cuda())
    torch.cuda.synchronize()
    got = tiles.cpu().numpy()
    assert got.shape == (ids.size, block, block, block)
    np.testing.assert_array_equal(got.view(np.uint8), want[ids].view(np.uint8))


def test_out_of_range_blocks_are_zero_and_flagged():
    import torch
    from paper_1903_07761_gb300 import cz
    f = _field((32, 32, 96), np.float32, seed=3)
    ref = O.compress(f, 32, O.W3AI, 1e-3)
    want = _blocks(O.decompress(ref), 32)
    st = torch.from_numpy(np.frombuffer(ref, np.uint8).copy()).cuda()
    ids = np.array([2, 3, -1, 0, 1], np.int32)
    ws = cz.Workspace()
    tiles = cz.decompress_blocks(st, torch.from_numpy(ids).cuda(), ws=ws, check=False)
    torch.cuda.synchronize()
    assert cz.cz_status(ws.buf.data_ptr(), torch.cuda.current_stream().cuda_stream) == cz.ERR_ARG
    got = tiles.cpu().numpy()
    assert not got[[1, 2]].any()  # indices 3 and -1 are outside the 3-block stream
    np.testing.assert_array_equal(got[0].view(np.uint32), want[2].view(np.uint32))
    np.testing.assert_array_equal(got[3].view(np.uint32), want[0].view(np.uint32))
    np.testing.assert_array_equal(got[4].view(np.uint32), want[1].view(np.uint32))


def test_empty_block_list_is_a_no_op():
    import torch
    from paper_1903_07761_gb300 import cz
    f = _field((32, 32, 32), np.float32, seed=4)
    ref = O.compress(f, 32, O.W3AI, 1e-3)
    st = torch.from_numpy(np.frombuffer(ref, np.uint8).copy()).cuda()
    tiles = cz.decompress_blocks(st, torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert tiles.shape == (0, 32, 32, 32)
