"""Quantities of a cell-struct array (cz_compress_aos): every chosen
component's stream equals the oracle's stream of that component as a dense
field, for mixed blocks, kinds and eps in one call."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


def _cells(shape, ncomp, dtype, seed):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64) for n in shape), indexing="ij")
    cells = np.empty(shape + (ncomp,))
    for c in range(ncomp):
        a, b = rng.uniform(2, 9, 2)
        cells[..., c] = (10 * c + 5) * (1 + 0.2 * np.sin(x / a) * np.cos(y / b) + 0.05 * np.sin(z / (a + b)))
        cells[..., c] += 1e-3 * rng.standard_normal(shape)
    return cells.astype(dtype)


@pytest.mark.parametrize("dtype,shape,ncomp", [
    (np.float32, (32, 64, 96), 7),
    (np.float64, (32, 32, 64), 5),
])
def test_each_component_stream_equals_the_oracle(dtype, shape, ncomp):
    import torch
    from paper_1903_07761_gb300 import cz
    cells = _cells(shape, ncomp, dtype, seed=ncomp)
    comps = [0, 3, ncomp - 1, 3]
    blocks = [32, 16, 32, 8] if dtype == np.float32 else [16, 32, 16, 8]
    kinds = ["w3ai", "w4", "w4li", "w3ai"]
    epss = [1e-3, 1e-2, 1e-4, 1e-3]
    res = cz.compress_aos(torch.from_numpy(cells).cuda(), comps, block=blocks, kind=kinds, eps=epss)
    torch.cuda.synchronize()
    for (out, nb), c, B, k, e in zip(res, comps, blocks, kinds, epss):
        got = out[:int(nb.item())].cpu().numpy().tobytes()
        field = np.ascontiguousarray(cells[..., c])
        assert got == O.compress(field, B, cz.KINDS[k], e)


def test_bad_components_and_mismatched_fields_are_refused():
    import torch
    from paper_1903_07761_gb300 import cz
    cells = torch.zeros((32, 32, 32, 4), device="cuda")
    with pytest.raises(cz.CzError) as e:
        cz.compress_aos(cells, [0, 4])
    assert e.value.code == cz.ERR_ARG
    with pytest.raises(cz.CzError) as e:
        cz.compress_aos(cells, [-1])
    assert e.value.code == cz.ERR_ARG
