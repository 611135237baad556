"""Out-of-bounds writes: every buffer the library writes (stream, field,
tiles, workspace) is allocated at exactly the size the API documents, with
guard bytes of a known pattern before and after it; after the call (and a
device synchronisation) the guards must be untouched.  Cases with the
largest payloads (eps = 0: every coefficient kept) and every block lane."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

GUARD = 4096
PAT = 0xA5


def _guarded(nbytes):
    """A uint8 CUDA buffer of nbytes between two guard zones; returns
    (inner view, whole buffer)."""
    import torch
    whole = torch.full((nbytes + 2 * GUARD,), PAT, dtype=torch.uint8, device="cuda")
    return whole[GUARD:GUARD + nbytes], whole


def _intact(whole):
    import torch
    torch.cuda.synchronize()
    g = torch.cat([whole[:GUARD], whole[-GUARD:]])
    return bool((g == PAT).all().item())


def _noise(shape, dtype, seed):
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)


LANES = [(np.float32, 8, (16, 16, 24)), (np.float32, 16, (32, 16, 48)), (np.float32, 32, (32, 64, 32)),
         (np.float64, 8, (8, 16, 24)), (np.float64, 16, (16, 32, 32)), (np.float64, 32, (32, 32, 64)),
         (np.float32, 64, (64, 64, 64))]


@pytest.mark.parametrize("stage2", [True, False])
@pytest.mark.parametrize("dtype,B,shape", LANES)
def test_compress_and_decompress_stay_inside_their_buffers(dtype, B, shape, stage2):
    import torch
    from paper_1903_07761_gb300 import cz
    f = _noise(shape, dtype, seed=B)
    ft = torch.from_numpy(f).cuda()
    p = cz.params_for(shape, dtype == np.float64, B, "w4li", 0.0, cz.EPS_REL, stage2, -1.0)
    cap = cz.cz_compress_bound(p)
    out, out_w = _guarded(cap)
    ws, ws_w = _guarded(cz.cz_workspace_size(p))
    nb, nb_w = _guarded(8)
    s = torch.cuda.current_stream().cuda_stream
    assert cz.cz_compress(p, ft.data_ptr(), out.data_ptr(), cap, nb.data_ptr(), ws.data_ptr(), ws.numel(), s) == cz.OK
    assert cz.cz_status(ws.data_ptr(), s) == cz.OK
    assert _intact(out_w) and _intact(ws_w) and _intact(nb_w)
    n = int(nb.view(torch.int64).item())
    stream = out[:n].cpu().numpy().tobytes()
    assert stream == O.compress(f, B, O.W4LI, 0.0, stage2=stage2)
    # decode into an exact-size field and an exact-size workspace
    fo, fo_w = _guarded(f.nbytes)
    ws2, ws2_w = _guarded(cz.cz_workspace_size(p))
    hdr = cz.C.create_string_buffer(stream[:cz.HEADER_BYTES], cz.HEADER_BYTES)
    assert cz.lib().cz_decompress(out.data_ptr(), n, hdr, fo.data_ptr(), f.nbytes, ws2.data_ptr(), ws2.numel(),
                                  s) == cz.OK
    assert cz.cz_status(ws2.data_ptr(), s) == cz.OK
    assert _intact(fo_w) and _intact(ws2_w)
    np.testing.assert_array_equal(fo.cpu().numpy().view(dtype).reshape(shape).view(np.uint8),
                                  O.decompress(stream).view(np.uint8))


@pytest.mark.parametrize("dtype,B,shape", [LANES[2], LANES[5], LANES[6]])
def test_random_access_and_cache_stay_inside_their_buffers(dtype, B, shape):
    import ctypes as C
    import torch
    from paper_1903_07761_gb300 import cz
    f = _noise(shape, dtype, seed=7)
    stream = O.compress(f, B, O.W3AI, 0.0)
    st = torch.from_numpy(np.frombuffer(stream, np.uint8).copy()).cuda()
    nblk = f.size // B ** 3
    ids = np.array([nblk - 1, 0, nblk - 1], np.int32)
    tile = B ** 3 * np.dtype(dtype).itemsize
    p, _ = cz.cz_read_header(stream)
    need = C.c_size_t()
    assert cz.lib().cz_decompress_blocks_workspace_size(C.byref(p), ids.size, C.byref(need)) == cz.OK
    tiles, tiles_w = _guarded(ids.size * tile)
    ws, ws_w = _guarded(need.value)
    hdr = C.create_string_buffer(stream[:cz.HEADER_BYTES], cz.HEADER_BYTES)
    d_ids = torch.from_numpy(ids).cuda()
    s = torch.cuda.current_stream().cuda_stream
    assert cz.lib().cz_decompress_blocks(st.data_ptr(), len(stream), hdr, d_ids.data_ptr(), ids.size,
                                         tiles.data_ptr(), ids.size * tile, ws.data_ptr(), ws.numel(), s) == cz.OK
    assert _intact(tiles_w) and _intact(ws_w)
    # the cache, with exact-size tiles and workspace
    c = cz.Cache(4, B, f64=dtype == np.float64)
    t2, t2_w = _guarded(ids.size * tile)
    ws3, ws3_w = _guarded(need.value)
    hits = C.c_int()
    for _ in range(2):
        assert cz.lib().cz_cache_fetch(c._h, st.data_ptr(), len(stream), hdr, ids.ctypes.data_as(C.c_void_p),
                                       ids.size, t2.data_ptr(), ids.size * tile, ws3.data_ptr(), ws3.numel(), s,
                                       C.byref(hits)) == cz.OK
    assert hits.value == 3
    assert _intact(t2_w) and _intact(ws3_w)
    np.testing.assert_array_equal(t2.cpu().numpy(), tiles.cpu().numpy())


def test_batch_and_cell_struct_outputs_stay_inside_their_buffers():
    import ctypes as C
    import torch
    from paper_1903_07761_gb300 import cz
    cells = _noise((32, 32, 64, 3), np.float32, seed=9)
    ct = torch.from_numpy(cells).cuda()
    comps = [2, 0]
    params = [cz.params_for((32, 32, 64), False, B, "w3ai", 0.0) for B in (32, 16)]
    arr = (cz.Params * 2)(*params)
    caps = [cz.cz_compress_bound(q) for q in params]
    outs = [_guarded(c) for c in caps]
    nbytes, nb_w = _guarded(16)
    need = C.c_size_t()
    assert cz.lib().cz_aos_workspace_size(2, arr, C.byref(need)) == cz.OK
    ws, ws_w = _guarded(need.value)
    s = torch.cuda.current_stream().cuda_stream
    comps_a = (C.c_int32 * 2)(*comps)
    assert cz.lib().cz_compress_aos(2, arr, ct.data_ptr(), 3, comps_a, (C.c_void_p * 2)(*[o.data_ptr() for o, _ in outs]),
                                    (C.c_size_t * 2)(*caps), nbytes.data_ptr(), ws.data_ptr(), ws.numel(), s) == cz.OK
    assert cz.cz_status(ws.data_ptr(), s) == cz.OK
    assert all(_intact(w) for _, w in outs) and _intact(nb_w) and _intact(ws_w)
    lens = nbytes.view(torch.int64).cpu().numpy()
    for i, ((o, _), c, B) in enumerate(zip(outs, comps, (32, 16))):
        got = o[:int(lens[i])].cpu().numpy().tobytes()
        assert got == O.compress(np.ascontiguousarray(cells[..., c]), B, O.W3AI, 0.0)


GROUP_LANES = [(np.float32, 8, 16, (16, 32, 48)), (np.float32, 16, 16, (32, 32, 64)),
               (np.float32, 32, 8, (32, 64, 96)), (np.float64, 16, 8, (16, 32, 64)),
               (np.float64, 32, 4, (32, 32, 96))]


@pytest.mark.parametrize("eps", [0.0, 1e-3])
@pytest.mark.parametrize("dtype,B,G,shape", GROUP_LANES)
def test_group_streams_stay_inside_their_buffers(dtype, B, G, shape, eps):
    """Aggregate chunks: eps = 0 sends the groups through the large-group
    tiers (global scratch), 1e-3 through the shared-memory ones; the decode
    and a random-access call use exact-size workspaces too."""
    import ctypes as C
    import torch
    from paper_1903_07761_gb300 import cz
    f = _noise(shape, dtype, seed=B + G)
    ft = torch.from_numpy(f).cuda()
    p = cz.params_for(shape, dtype == np.float64, B, "w3ai", eps, cz.EPS_REL, True, -1.0, group=G)
    cap = cz.cz_compress_bound(p)
    out, out_w = _guarded(cap)
    ws, ws_w = _guarded(cz.cz_workspace_size(p))
    nb, nb_w = _guarded(8)
    s = torch.cuda.current_stream().cuda_stream
    assert cz.cz_compress(p, ft.data_ptr(), out.data_ptr(), cap, nb.data_ptr(), ws.data_ptr(), ws.numel(), s) == cz.OK
    assert cz.cz_status(ws.data_ptr(), s) == cz.OK
    assert _intact(out_w) and _intact(ws_w) and _intact(nb_w)
    n = int(nb.view(torch.int64).item())
    stream = out[:n].cpu().numpy().tobytes()
    assert stream == O.compress(f, B, O.W3AI, eps, group=G)
    want = O.decompress(stream)
    hdr = cz.C.create_string_buffer(stream[:cz.HEADER_BYTES], cz.HEADER_BYTES)
    need = C.c_size_t()
    assert cz.lib().cz_decompress_blocks_workspace_size(C.byref(p), f.size // B ** 3, C.byref(need)) == cz.OK
    fo, fo_w = _guarded(f.nbytes)
    ws2, ws2_w = _guarded(need.value)
    assert cz.lib().cz_decompress(out.data_ptr(), n, hdr, fo.data_ptr(), f.nbytes, ws2.data_ptr(), ws2.numel(),
                                  s) == cz.OK
    assert cz.cz_status(ws2.data_ptr(), s) == cz.OK
    assert _intact(fo_w) and _intact(ws2_w)
    np.testing.assert_array_equal(fo.cpu().numpy().view(dtype).reshape(shape).view(np.uint8), want.view(np.uint8))
    ids = torch.tensor([f.size // B ** 3 - 1, 0, 1], dtype=torch.int32, device="cuda")
    assert cz.lib().cz_decompress_blocks_workspace_size(C.byref(p), 3, C.byref(need)) == cz.OK
    tl, tl_w = _guarded(3 * B ** 3 * f.itemsize)
    ws3, ws3_w = _guarded(need.value)
    assert cz.lib().cz_decompress_blocks(out.data_ptr(), n, hdr, ids.data_ptr(), 3, tl.data_ptr(), tl.numel(),
                                         ws3.data_ptr(), ws3.numel(), s) == cz.OK
    assert cz.cz_status(ws3.data_ptr(), s) == cz.OK
    assert _intact(tl_w) and _intact(ws3_w)
