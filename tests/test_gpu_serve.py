"""The request server: compress and decompress requests of mixed sizes and
precisions submitted back to back must give the same bytes as the same
calls made alone, while the server admits them under its memory budget,
batches compatible compress requests and overlaps work on several streams.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _mix(seed, n=24, f64_block=16):
    from paper_1903_07761_gb300 import inputs
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        f64 = rng.random() < 0.3
        e = int(32 * rng.integers(1, 5))
        dims = (e, e, e)
        f = inputs.field(inputs.P, dims, np.float64 if f64 else np.float32, seed=4000 + i, nbubbles=4)
        out.append((f, f64_block if f64 else 32, float(rng.choice([1e-3, 1e-4])), "w3ai" if i % 2 else "w4"))
    return out


def _alone(cz, torch, t, B, e, kind):
    out, nb = cz.compress(t, block=B, kind=kind, eps=e)
    torch.cuda.synchronize()
    return out[:int(nb.item())].cpu().numpy().tobytes()


@pytest.mark.parametrize("budget_mib,streams,f64_block", [(2048, 4, 16), (96, 2, 16), (2048, 4, 32)])
def test_mixed_requests_equal_alone(budget_mib, streams, f64_block):
    """f64_block = 32: the FP64 requests take 32^3 blocks (the slab kernels)."""
    import torch
    from paper_1903_07761_gb300 import cz
    items = _mix(1, f64_block=f64_block)
    tens = [torch.from_numpy(f).cuda() for f, _, _, _ in items]
    alone = [_alone(cz, torch, t, B, e, k) for t, (_, B, e, k) in zip(tens, items)]
    # decompress requests of the first few streams, mixed in
    dec_in = []
    for s in alone[:6]:
        d = torch.from_numpy(np.frombuffer(s, np.uint8).copy()).cuda()
        dec_in.append((d, len(s), s[:cz.HEADER_BYTES]))
    dec_alone = [cz.decompress(d, nbytes=n).cpu().numpy() for d, n, _ in dec_in]
    torch.cuda.synchronize()
    outs, lens, tickets = [], [], []
    dec_out = []
    with cz.Server(budget_mib << 20, streams) as srv:
        for i, (t, (_, B, e, k)) in enumerate(zip(tens, items)):
            p = cz.params_for(tuple(t.shape), t.dtype == torch.float64, B, k, e)
            cap = cz.cz_compress_bound(p)
            o = torch.zeros(cap, dtype=torch.uint8, device="cuda")
            nb = torch.zeros(1, dtype=torch.int64, device="cuda")
            outs.append(o)
            lens.append(nb)
            tickets.append(("c", i, srv.submit_compress(p, t.data_ptr(), o.data_ptr(), cap, nb.data_ptr())))
            if i < len(dec_in):
                d, n, h = dec_in[i]
                ref = dec_alone[i]
                fo = torch.zeros(ref.size, dtype=torch.float64 if ref.dtype == np.float64 else torch.float32,
                                 device="cuda")
                dec_out.append(fo)
                tickets.append(("d", i, srv.submit_decompress(d.data_ptr(), n, h, fo.data_ptr(),
                                                              fo.numel() * fo.element_size())))
        lat = []
        for kind, i, tk in tickets:
            res, ms = srv.wait(tk)
            assert res == cz.OK
            assert ms >= 0
            lat.append(ms)
    torch.cuda.synchronize()
    for i in range(len(items)):
        got = outs[i][:int(lens[i].item())].cpu().numpy().tobytes()
        assert got == alone[i]
    for i, fo in enumerate(dec_out):
        np.testing.assert_array_equal(fo.cpu().numpy().reshape(dec_alone[i].shape).view(np.uint8),
                                      dec_alone[i].view(np.uint8))


def test_request_beyond_budget_is_refused():
    import torch
    from paper_1903_07761_gb300 import cz
    t = torch.zeros((256, 256, 256), device="cuda")
    p = cz.params_for(tuple(t.shape), False, 32, "w4", 1e-3)
    with cz.Server(4 << 20, 1) as srv:
        with pytest.raises(cz.CzError) as e:
            srv.submit_compress(p, t.data_ptr(), t.data_ptr(), 1 << 20, 0)
        assert e.value.code == cz.ERR_BUDGET
