"""Host- and device-side error reporting of the C ABI (no GPU fault).

Bad parameters are refused on the host; a too-small output buffer and a
corrupted stream are reported through the workspace status word while the
kernels finish normally (they never trap).  Corrupted streams are made on the
host.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


def _field(shape=(32, 32, 64), dtype=np.float32):
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64) for n in shape), indexing="ij")
    return (np.sin(x / 4) + np.cos(y / 6) * z / 10).astype(dtype)


def test_bad_parameters_are_refused():
    import torch
    from paper_1903_07761_gb300 import cz
    f = torch.zeros((32, 32, 48), device="cuda")  # 48 not a multiple of 32
    with pytest.raises(cz.CzError) as e:
        cz.compress(f, block=32)
    assert e.value.code == cz.ERR_ARG
    with pytest.raises(cz.CzError):
        cz.compress(torch.zeros((16, 16, 16), device="cuda"), block=12)
    with pytest.raises(cz.CzError):
        cz.compress(torch.zeros((16, 16, 16), device="cuda"), block=16, eps=-1.0)


def test_output_capacity_too_small_sets_status():
    import torch
    from paper_1903_07761_gb300 import cz
    f = torch.from_numpy(_field()).cuda()
    p = cz.params_for(tuple(f.shape), False, 32, cz.W4, 0.0)
    need = cz.cz_compress_bound(p)
    ws = torch.empty(cz.cz_workspace_size(p), dtype=torch.uint8, device="cuda")
    out = torch.zeros(need, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    # header + table fits, chunks do not
    cap = 1024
    assert cz.cz_compress(p, f.data_ptr(), out.data_ptr(), cap, nb.data_ptr(), ws.data_ptr(),
                          ws.numel(), s) == cz.OK
    assert cz.cz_status(ws.data_ptr(), s) == cz.ERR_CAPACITY
    assert int(nb.item()) > cap  # the size that would be needed
    assert int(out[cap:].sum().item()) == 0  # nothing written past the capacity
    # below the fixed header + table size the host refuses
    assert cz.cz_compress(p, f.data_ptr(), out.data_ptr(), 64, nb.data_ptr(), ws.data_ptr(),
                          ws.numel(), s) == cz.ERR_CAPACITY
    # too small workspace
    assert cz.cz_compress(p, f.data_ptr(), out.data_ptr(), need, nb.data_ptr(), ws.data_ptr(),
                          16, s) == cz.ERR_CAPACITY


@pytest.mark.parametrize("stage2", [True, False])
def test_corrupt_stream_sets_status_and_zeroes_block(stage2):
    import torch
    from paper_1903_07761_gb300 import cz
    f = _field()
    ref = bytearray(O.compress(f, 32, O.W3AI, 1e-3, stage2=stage2))
    data0, offs = O.chunk_table(bytes(ref))
    bad = bytearray(ref)
    c1 = data0 + int(offs[1])
    bad[c1:c1 + 4] = (32 ** 3).to_bytes(4, "little")  # nnz too large in block 1
    s = torch.from_numpy(np.frombuffer(bytes(bad), np.uint8).copy()).cuda()
    with pytest.raises(cz.CzError) as e:
        cz.decompress(s, nbytes=len(bad))
    assert e.value.code == cz.ERR_CORRUPT
    out = cz.decompress(s, nbytes=len(bad), check=False)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.all(o[:, :, 32:64] == 0)  # block 1 written as zeros
    np.testing.assert_array_equal(o[:, :, :32], O.decompress(bytes(ref))[:, :, :32])


def test_corrupt_tokens_and_offsets():
    import torch
    from paper_1903_07761_gb300 import cz
    f = _field()
    ref = bytearray(O.compress(f, 32, O.W4, 1e-3, stage2=True))
    data0, offs = O.chunk_table(bytes(ref))
    for mutate in ("token", "offset"):
        bad = bytearray(ref)
        if mutate == "token":
            t0 = data0 + int(offs[0]) + 8
            bad[t0:t0 + 4] = (0xFFFF | (0x7FFF << 16)).to_bytes(4, "little")
        else:
            bad[O.HEADER_BYTES + 8:O.HEADER_BYTES + 16] = (10 ** 9).to_bytes(8, "little")
        s = torch.from_numpy(np.frombuffer(bytes(bad), np.uint8).copy()).cuda()
        with pytest.raises(cz.CzError) as e:
            cz.decompress(s, nbytes=len(bad))
        assert e.value.code == cz.ERR_CORRUPT, mutate
    # a truncated stream is refused on the host
    s = torch.from_numpy(np.frombuffer(bytes(ref), np.uint8).copy()).cuda()
    with pytest.raises(cz.CzError) as e:
        cz.decompress(s, nbytes=len(ref) - 4)
    assert e.value.code == cz.ERR_CORRUPT


def test_repeated_runs_are_deterministic():
    f = _field((64, 32, 64))
    from gpu_helpers import gpu_compress
    a = gpu_compress(f, 16, O.W4LI, 1e-3)
    b = gpu_compress(f, 16, O.W4LI, 1e-3)
    assert a == b
