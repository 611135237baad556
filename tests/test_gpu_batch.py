"""Batched compression: many fields of uneven block counts, mixed FP32 /
FP64, per-field eps, in one call.  Every field's stream must equal, byte for
byte, the one cz_compress writes for it alone (and hence the oracle's), also
after the autotuner has picked its launch shape and when the call is
replayed from a captured CUDA graph.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


def _fields(seed, n=12):
    from paper_1903_07761_gb300 import inputs
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        f64 = bool(i % 3 == 2)
        B = 16 if f64 else 32
        dims = tuple(int(B * rng.integers(1, 4)) for _ in range(3))
        f = inputs.field(inputs.P, dims, np.float64 if f64 else np.float32, seed=3000 + i, nbubbles=6)
        out.append((f, B, float(rng.choice([1e-2, 1e-3, 1e-4]))))
    return out


def test_batch_streams_equal_single_field_streams():
    import torch
    from paper_1903_07761_gb300 import cz
    items = _fields(1)
    tens = [torch.from_numpy(f).cuda() for f, _, _ in items]
    res = cz.compress_batch(tens, block=[B for _, B, _ in items], kind="w3ai",
                            eps=[e for _, _, e in items])
    torch.cuda.synchronize()
    for (f, B, e), t, (out, nb) in zip(items, tens, res):
        single, snb = cz.compress(t, block=B, kind="w3ai", eps=e)
        torch.cuda.synchronize()
        got = out[:int(nb.item())].cpu().numpy().tobytes()
        want = single[:int(snb.item())].cpu().numpy().tobytes()
        assert got == want
    # and the oracle agrees on a few of them
    for (f, B, e), (out, nb) in list(zip(items, res))[:4]:
        got = out[:int(nb.item())].cpu().numpy().tobytes()
        assert got == O.compress(f, B, O.W3AI, e)


@pytest.mark.parametrize("kind", ["w4", "w4li"])
def test_batch_other_kinds_and_strict(kind):
    import torch
    from paper_1903_07761_gb300 import cz
    items = _fields(2, n=6)
    tens = [torch.from_numpy(f).cuda() for f, _, _ in items]
    for bm in (cz.BOUND_PAPER, cz.BOUND_STRICT):
        res = cz.compress_batch(tens, kind=kind, eps=[e for _, _, e in items], bound_mode=bm)
        torch.cuda.synchronize()
        for (f, B, e), (out, nb) in zip(items, res):
            got = out[:int(nb.item())].cpu().numpy().tobytes()
            assert got == O.compress(f, B, cz.KINDS[kind], e, bound_mode=bm)


def test_batch_tuned_and_graph_replay_give_the_same_streams():
    import torch
    from paper_1903_07761_gb300 import cz
    items = _fields(3, n=10)
    tens = [torch.from_numpy(f).cuda() for f, _, _ in items]
    ref = [bytes(o[:int(n.item())].cpu().numpy()) for o, n in
           cz.compress_batch(tens, kind="w3ai", eps=[e for _, _, e in items])]
    # tuned launch shape
    res = cz.compress_batch(tens, kind="w3ai", eps=[e for _, _, e in items], tune=True)
    torch.cuda.synchronize()
    assert [bytes(o[:int(n.item())].cpu().numpy()) for o, n in res] == ref
    # captured in a CUDA graph (set up by one call outside the capture)
    params, caps, outs = [], [], []
    for (f, B, e), t in zip(items, tens):
        p = cz.params_for(tuple(t.shape), t.dtype == torch.float64, B, "w3ai", e)
        params.append(p)
        caps.append(cz.cz_compress_bound(p))
        outs.append(torch.zeros(caps[-1], dtype=torch.uint8, device="cuda"))
    nbytes = torch.zeros(len(items), dtype=torch.int64, device="cuda")
    ws = torch.empty(cz.cz_batch_workspace_size(params), dtype=torch.uint8, device="cuda")
    b = cz.BatchArgs(params, [t.data_ptr() for t in tens], [o.data_ptr() for o in outs], caps)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        assert cz.cz_compress_batch(b, nbytes.data_ptr(), ws.data_ptr(), ws.numel(), side.cuda_stream) == cz.OK
    torch.cuda.synchronize()
    for o in outs:
        o.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        assert cz.cz_compress_batch(b, nbytes.data_ptr(), ws.data_ptr(), ws.numel(),
                                    torch.cuda.current_stream().cuda_stream) == cz.OK
    for _ in range(2):
        for o in outs:
            o.zero_()
        nbytes.zero_()
        g.replay()
        torch.cuda.synchronize()
        got = [bytes(o[:int(n)].cpu().numpy()) for o, n in zip(outs, nbytes.cpu().tolist())]
        assert got == ref


def test_batch_with_bit_zeroing_groups_and_matches_the_oracle():
    """Fields with and without bit zeroing in one batch: each stream equals
    the oracle's with the same zeroing width."""
    import torch
    from paper_1903_07761_gb300 import cz
    items = _fields(11, n=4)
    zb = [8, 0, 4, 8]
    tens = [torch.from_numpy(f).cuda() for f, _, _ in items]
    params, caps, outs = [], [], []
    for (f, B, e), t, z in zip(items, tens, zb):
        p = cz.params_for(tuple(t.shape), t.dtype == torch.float64, B, "w3ai", e, zero_bits=z)
        params.append(p)
        caps.append(cz.cz_compress_bound(p))
        outs.append(torch.zeros(caps[-1], dtype=torch.uint8, device="cuda"))
    nbytes = torch.zeros(len(items), dtype=torch.int64, device="cuda")
    ws = torch.empty(cz.cz_batch_workspace_size(params), dtype=torch.uint8, device="cuda")
    b = cz.BatchArgs(params, [t.data_ptr() for t in tens], [o.data_ptr() for o in outs], caps)
    s = torch.cuda.current_stream().cuda_stream
    assert cz.cz_compress_batch(b, nbytes.data_ptr(), ws.data_ptr(), ws.numel(), s) == cz.OK
    torch.cuda.synchronize()
    for (f, B, e), o, n, z in zip(items, outs, nbytes.cpu().tolist(), zb):
        assert bytes(o[:int(n)].cpu().numpy()) == O.compress(f, B, O.W3AI, e, zbits=z)


def test_batch_with_fp64_32_blocks_matches_the_oracle():
    """FP64 fields with 32^3 blocks (the slab kernels) in one batched call,
    next to FP32 fields: every stream equals the oracle's."""
    import torch
    from paper_1903_07761_gb300 import cz, inputs
    rng = np.random.default_rng(41)
    items = []
    for i in range(5):
        f64 = i % 2 == 0
        dims = tuple(int(32 * rng.integers(1, 3)) for _ in range(3))
        f = inputs.field(inputs.P, dims, np.float64 if f64 else np.float32, seed=3100 + i, nbubbles=4)
        items.append((f, float(rng.choice([1e-2, 1e-3, 1e-4]))))
    tens = [torch.from_numpy(f).cuda() for f, _ in items]
    res = cz.compress_batch(tens, block=32, kind="w3ai", eps=[e for _, e in items])
    torch.cuda.synchronize()
    for (f, e), (out, nb) in zip(items, res):
        got = out[:int(nb.item())].cpu().numpy().tobytes()
        assert got == O.compress(f, 32, O.W3AI, e)


@pytest.mark.parametrize("kind", ["w3ai", "w4li"])
def test_every_tuner_setting_gives_the_same_streams(kind):
    """Every knob setting the tuner may pick -- stage kernel family (FP32
    32^3: the block in registers or in global scratch), stage grid, stage-2
    grid, look-back tile of 64 / 128 / 256 chunks -- writes the streams that
    cz_compress writes for each field alone (and hence the oracle's)."""
    import ctypes as C
    import itertools
    import torch
    from paper_1903_07761_gb300 import cz
    items = _fields(5, n=9)
    tens = [torch.from_numpy(f).cuda() for f, _, _ in items]
    params, caps, outs, ref = [], [], [], []
    for (f, B, e), t in zip(items, tens):
        p = cz.params_for(tuple(t.shape), t.dtype == torch.float64, B, kind, e)
        params.append(p)
        caps.append(cz.cz_compress_bound(p))
        outs.append(torch.zeros(caps[-1], dtype=torch.uint8, device="cuda"))
        single, snb = cz.compress(t, block=B, kind=kind, eps=e)
        ref.append(single[:int(snb.item())].cpu().numpy().tobytes())
    nbytes = torch.zeros(len(items), dtype=torch.int64, device="cuda")
    ws = torch.empty(cz.cz_batch_workspace_size(params), dtype=torch.uint8, device="cuda")
    b = cz.BatchArgs(params, [t.data_ptr() for t in tens], [o.data_ptr() for o in outs], caps)
    L = cz.lib()
    L.czi_compress_batch_knobs.argtypes = [C.c_int, C.POINTER(cz.Params), C.POINTER(C.c_void_p),
                                           C.POINTER(C.c_void_p), C.POINTER(C.c_size_t), C.c_void_p, C.c_void_p,
                                           C.c_size_t, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int]
    L.czi_compress_batch_knobs.restype = C.c_int
    s = torch.cuda.current_stream().cuda_stream
    for slab, s1, s2, pt in itertools.product((0, 1), (0, 1), (1, 2), (64, 128, 256)):
        for o in outs:
            o.fill_(0xA5)
        r = L.czi_compress_batch_knobs(b.n, b.params, b.fields, b.outs, b.caps, nbytes.data_ptr(), ws.data_ptr(),
                                       ws.numel(), s, s1, s2, pt, slab)
        assert r == cz.OK
        assert cz.cz_status(ws.data_ptr(), s) == cz.OK
        got = [bytes(o[:int(n)].cpu().numpy()) for o, n in zip(outs, nbytes.cpu().tolist())]
        assert got == ref, (slab, s1, s2, pt)
