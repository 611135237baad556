"""cz_compress_noalloc: the compress entry point with the library's own
fixed workspace.  Its streams must equal those of cz_compress with a
caller-supplied workspace, call after call, and fields whose workspace
exceeds the fixed size must be refused on the host.

Collected last, so that it runs both alone and after every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _stream_with_workspace(cz, torch, f, p, cap, s):
    out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(cz.cz_workspace_size(p), dtype=torch.uint8, device="cuda")
    r = cz.cz_compress(p, f.data_ptr(), out.data_ptr(), cap, nb.data_ptr(), ws.data_ptr(), ws.numel(), s)
    assert r == cz.OK
    assert cz.cz_status(ws.data_ptr(), s) == cz.OK
    n = int(nb.item())
    return out[:n].cpu().numpy().tobytes()


@pytest.mark.parametrize("kind,stage2,range_", [("w4", True, -1.0), ("w3ai", False, -1.0), ("w4li", True, 250.0)])
def test_noalloc_matches_workspace_entry_point(kind, stage2, range_):
    import torch
    from paper_1903_07761_gb300 import cz, inputs
    f = torch.from_numpy(inputs.config0(seed=0)).cuda()
    s = torch.cuda.current_stream().cuda_stream
    p = cz.params_for(tuple(f.shape), False, 32, kind, 1e-3, cz.EPS_REL, stage2, range_)
    need = cz.cz_workspace_size(p)
    assert need <= cz.NOALLOC_WS_BYTES
    cap = cz.cz_compress_bound(p)
    ref = _stream_with_workspace(cz, torch, f, p, cap, s)
    for _ in range(2):  # two calls in a row reuse the same fixed workspace
        out = torch.full((cap,), 0xA5, dtype=torch.uint8, device="cuda")
        nb = torch.zeros(1, dtype=torch.int64, device="cuda")
        r = cz.cz_compress_noalloc(p, f.data_ptr(), out.data_ptr(), cap, nb.data_ptr(), s)
        assert r == cz.OK
        assert cz.cz_noalloc_status(s) == cz.OK
        torch.cuda.synchronize()
        n = int(nb.item())
        got = out[:n].cpu().numpy().tobytes()
        assert n == len(ref)
        assert got == ref


def test_noalloc_refuses_fields_beyond_its_workspace():
    import torch
    from paper_1903_07761_gb300 import cz
    p = cz.params_for((512, 512, 512), False, 32, "w4", 1e-3, cz.EPS_REL, True, 1.0)
    assert cz.cz_workspace_size(p) > cz.NOALLOC_WS_BYTES
    # refused on the host before anything is enqueued: the buffers are not touched
    small = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(16, dtype=torch.uint8, device="cuda")
    r = cz.cz_compress_noalloc(p, small.data_ptr(), out.data_ptr(), out.numel(), 0,
                               torch.cuda.current_stream().cuda_stream)
    assert r == cz.ERR_CAPACITY
    torch.cuda.synchronize()
    assert int(out.sum().item()) == 0


def test_noalloc_output_too_small_reports_length_and_status():
    import torch
    from paper_1903_07761_gb300 import cz, inputs
    f = torch.from_numpy(inputs.config0(seed=1)).cuda()
    s = torch.cuda.current_stream().cuda_stream
    p = cz.params_for(tuple(f.shape), False, 32, "w4", 1e-3, cz.EPS_REL, True, -1.0)
    cap = cz.cz_compress_bound(p)
    full = _stream_with_workspace(cz, torch, f, p, cap, s)
    small = len(full) // 2
    out = torch.zeros(small, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert cz.cz_compress_noalloc(p, f.data_ptr(), out.data_ptr(), small, nb.data_ptr(), s) == cz.OK
    # the device status word of that call, kept in the library's array
    assert cz.cz_noalloc_status(s) == cz.ERR_CAPACITY
    torch.cuda.synchronize()
    assert int(nb.item()) == len(full) > small
    np.testing.assert_array_equal(out[:cz.HEADER_BYTES].cpu().numpy(),
                                  np.frombuffer(full[:cz.HEADER_BYTES], np.uint8))
    # the next call that fits clears it
    out2 = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    assert cz.cz_compress_noalloc(p, f.data_ptr(), out2.data_ptr(), cap, nb.data_ptr(), s) == cz.OK
    assert cz.cz_noalloc_status(s) == cz.OK
    assert out2[:int(nb.item())].cpu().numpy().tobytes() == full
