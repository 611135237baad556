"""Decoded-block cache (cz_cache_*): blocks served from the cache and blocks
decoded on a miss are exactly the oracle's decoded blocks; the cache keeps
the least recently used order, decodes each missing block once per call,
starts over for another stream and refuses bad requests on the host."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


def _field(shape, dtype, seed):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64) for n in shape), indexing="ij")
    f = 30 + 10 * np.sin(x / 5.3 + rng.random()) * np.cos(y / 3.9) + 2 * np.sin(z / 2.7)
    f += 1e-3 * rng.standard_normal(shape)
    return f.astype(dtype)


def _blocks(field, B):
    nz, ny, nx = (n // B for n in field.shape)
    return field.reshape(nz, B, ny, B, nx, B).transpose(0, 2, 4, 1, 3, 5).reshape(-1, B, B, B)


def _stream(dtype, B, shape, seed, kind=O.W3AI, stage2=True):
    import torch
    f = _field(shape, dtype, seed)
    ref = O.compress(f, B, kind, 1e-3, stage2=stage2)
    want = _blocks(O.decompress(ref), B)
    st = torch.from_numpy(np.frombuffer(ref, np.uint8).copy()).cuda()
    return st, want


@pytest.mark.parametrize("dtype,B,shape", [
    (np.float32, 32, (32, 96, 128)),   # 12 blocks
    (np.float64, 16, (32, 32, 48)),    # 12 blocks
    (np.float32, 8, (16, 16, 24)),     # 12 blocks
])
def test_hits_misses_and_lru_order(dtype, B, shape):
    import torch
    from paper_1903_07761_gb300 import cz
    st, want = _stream(dtype, B, shape, seed=B)
    c = cz.Cache(4, B, f64=dtype == np.float64)
    # (request, hits expected): LRU order after each call, most recent first
    steps = [
        ([0, 5, 3], 0),        # decode 0 5 3                     -> 3 5 0
        ([5, 7, 0, 0], 3),     # 5, 0, 0 held; decode 7           -> 0 7 5 3
        ([9], 0),              # decode 9, replaces 3 (LRU)        -> 9 0 7 5
        ([3], 0),              # 3 was replaced: decode, replaces 5 -> 3 9 0 7
        ([5, 5, 11, 0], 1),    # 0 held; decode 5 and 11 (each once), replacing 7 and 9
        ([3, 5, 11, 0], 4),    # all held
    ]
    for ids, hits in steps:
        tiles, h = c.fetch(st, ids)
        torch.cuda.synchronize()
        assert h == hits, (ids, h)
        np.testing.assert_array_equal(tiles.cpu().numpy().view(np.uint8), want[ids].view(np.uint8))
    held, hits_tot, misses_tot = c.stats()
    assert held == 4
    assert hits_tot == sum(h for _, h in steps)
    assert misses_tot == 3 + 1 + 1 + 1 + 2 + 0
    c.close()


def test_another_stream_empties_the_cache_and_clear():
    import torch
    from paper_1903_07761_gb300 import cz
    st1, want1 = _stream(np.float32, 32, (32, 64, 64), seed=1)
    st2, want2 = _stream(np.float32, 32, (32, 64, 64), seed=2)
    c = cz.Cache(4, 32)
    t, h = c.fetch(st1, [0, 1, 2])
    assert h == 0
    t, h = c.fetch(st1, [2, 1])
    assert h == 2
    t, h = c.fetch(st2, [2, 1])  # same block ids, another stream: nothing held
    torch.cuda.synchronize()
    assert h == 0
    np.testing.assert_array_equal(t.cpu().numpy().view(np.uint8), want2[[2, 1]].view(np.uint8))
    c.clear()
    t, h = c.fetch(st2, [1])
    torch.cuda.synchronize()
    assert h == 0 and c.stats()[0] == 1
    np.testing.assert_array_equal(t.cpu().numpy().view(np.uint8), want2[[1]].view(np.uint8))


def test_stage2_off_and_every_kind():
    import torch
    from paper_1903_07761_gb300 import cz
    for kind in (O.W4, O.W4LI, O.W3AI):
        for stage2 in (True, False):
            st, want = _stream(np.float32, 16, (16, 32, 48), seed=10 + kind, kind=kind, stage2=stage2)
            c = cz.Cache(6, 16)
            rng = np.random.default_rng(kind)
            for _ in range(5):
                ids = rng.integers(0, want.shape[0], 6).tolist()
                t, h = c.fetch(st, ids)
                torch.cuda.synchronize()
                np.testing.assert_array_equal(t.cpu().numpy().view(np.uint8), want[ids].view(np.uint8))
            c.close()


def test_bad_requests_are_refused_on_the_host():
    from paper_1903_07761_gb300 import cz
    st, want = _stream(np.float32, 32, (32, 32, 96), seed=4)  # 3 blocks
    c = cz.Cache(2, 32)
    for ids in ([0, 1, 2], [3], [-1]):  # more than the capacity; out of range
        with pytest.raises(cz.CzError) as e:
            c.fetch(st, ids)
        assert e.value.code == cz.ERR_ARG
    assert c.stats() == (0, 0, 0)  # nothing was enqueued or kept
    c64 = cz.Cache(2, 32, f64=True)  # another element type than the stream's
    with pytest.raises(cz.CzError) as e:
        c64.fetch(st, [0])
    assert e.value.code == cz.ERR_ARG
    with pytest.raises(cz.CzError):
        cz.Cache(0, 32)
    with pytest.raises(cz.CzError):
        cz.Cache(4, 12)


def test_a_call_served_wholly_from_the_cache_resets_the_status_word():
    """A fetch whose blocks are all held decodes nothing; it still resets
    the status word of its workspace, so a workspace that held anything
    before (here: every byte 0xAB) reports success."""
    import torch
    from paper_1903_07761_gb300 import cz
    st, want = _stream(np.float32, 16, (16, 32, 32), seed=21)
    c = cz.Cache(4, 16)
    c.fetch(st, [0, 3])
    ws = cz.Workspace()
    ws.get(1 << 20).fill_(0xAB)
    t, h = c.fetch(st, [3, 0, 3], ws=ws)  # raises on a bad status word
    torch.cuda.synchronize()
    assert h == 3
    assert cz.cz_status(ws.buf.data_ptr(), torch.cuda.current_stream().cuda_stream) == cz.OK
    np.testing.assert_array_equal(t.cpu().numpy().view(np.uint8), want[[3, 0, 3]].view(np.uint8))
