"""Bounded device-side waits run out and report CZ_ERR_TIMEOUT.

The codec kernels wait in two ways: the look-back of the chunk-offset scan
spins on the state words of earlier tiles, and the stage and decode kernels
wait on an mbarrier for their TMA / bulk copies.  Both waits have an
iteration limit; on reaching it a kernel records CZ_ERR_TIMEOUT in its status
word and returns (it never traps).  A test-only probe (czi_wait_probe) runs
the same wait helpers with a short limit where the wait cannot end:
  * a tile that never publishes its aggregate (its state word stays 0), so
    the tiles after it spin until the limit;
  * an mbarrier armed for 16 bytes that no copy delivers (no copy is started,
    so nothing is left in flight when the CTA returns), where every thread
    gives up and the CTA decides at one barrier, as the codec kernels do.
Nothing here faults the GPU or waits without bound.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _probe(which, tiles, skip, limit):
    import torch
    from paper_1903_07761_gb300 import cz
    L = cz.lib()
    L.czi_wait_probe.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p]
    L.czi_wait_probe.restype = C.c_int
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    state = torch.zeros(tiles, dtype=torch.int64, device="cuda")
    out = torch.full((tiles,), -1, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    r = L.czi_wait_probe(which, tiles, skip, limit, status.data_ptr(), state.data_ptr(), out.data_ptr(), s)
    assert r == cz.OK
    torch.cuda.synchronize()  # the kernel ends by itself
    return int(status.item()), out.cpu().numpy()


def test_lookback_gives_up_when_a_tile_never_publishes():
    from paper_1903_07761_gb300 import cz
    tiles, skip = 12, 5
    st, out = _probe(0, tiles, skip, 1 << 12)
    assert st == cz.ERR_TIMEOUT
    # the tiles before the missing one got their exact prefixes (one per tile)
    np.testing.assert_array_equal(out[:skip], np.arange(skip))
    assert out[skip] == -1  # the missing tile wrote nothing


def test_lookback_completes_when_every_tile_publishes():
    from paper_1903_07761_gb300 import cz
    tiles = 40  # more than a warp's window of 32 predecessors
    st, out = _probe(0, tiles, tiles, 1 << 12)
    assert st == cz.OK
    np.testing.assert_array_equal(out, np.arange(tiles))


@pytest.mark.parametrize("threads", [32, 512])
def test_mbarrier_wait_gives_up_as_one_cta(threads):
    from paper_1903_07761_gb300 import cz
    st, out = _probe(1, threads, 0, 1 << 10)
    assert st == cz.ERR_TIMEOUT
    assert (out == 1).all()  # every thread saw the same decision
