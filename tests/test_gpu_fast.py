"""The fast build (CZ_FLAG_FAST): the compiler may fuse multiply-adds, so
coefficients move by a few ulps and the streams are no longer those of the
exact build.  It serves W3ai only (W4 and W4li are refused on the host:
their extrapolating rows flip enough keep/drop decisions to miss the PSNR
gate).  The gates, against the CPU oracle:
  * every coefficient within 2^-20 of the field range of the oracle's;
  * PSNR within 0.01 dB of the oracle's, compression factor within 1 %;
  * in strict bound mode, a decoded error of at most eps * range (plus the
    rounding of the reconstruction itself);
  * the stream header records the build, and decompression uses it.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

KINDS = (O.W3AI,)  # the kinds the fast build serves
CASES = [(np.float32, 32, (64, 64, 96)), (np.float32, 16, (32, 48, 64)), (np.float64, 16, (32, 32, 48))]
# the slab lanes (FP64 32^3, FP32 64^3) have a fast build too; a field of a
# few of their blocks is enough for the per-coefficient gate
COEF_CASES = CASES + [(np.float64, 32, (32, 32, 64)), (np.float32, 64, (64, 64, 64))]


def _field(shape, dtype, seed=5):
    from paper_1903_07761_gb300 import inputs
    return inputs.field(inputs.P, shape, dtype, seed=seed, nbubbles=8)


def _dense(cz, torch, f, block, kind, fast):
    t = torch.from_numpy(f).cuda()
    c = torch.empty_like(t)
    p = cz.params_for(f.shape, f.dtype == np.float64, block, kind, 1e-3, fast=fast)
    assert cz.cz_forward_dense(p, t.data_ptr(), c.data_ptr(), torch.cuda.current_stream().cuda_stream) == cz.OK
    torch.cuda.synchronize()
    return c.cpu().numpy().astype(np.float64)


def _blocks(shape, block):
    nz, ny, nx = shape
    for bz in range(nz // block):
        for by in range(ny // block):
            for bx in range(nx // block):
                yield np.s_[bz * block:(bz + 1) * block, by * block:(by + 1) * block, bx * block:(bx + 1) * block]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype,block,shape", COEF_CASES)
def test_fast_coefficients_close_to_the_oracle(dtype, block, shape, kind):
    """Every coefficient within 2^-20 of the field range of the oracle's."""
    import torch
    from paper_1903_07761_gb300 import cz
    f = _field(shape, dtype)
    fast = _dense(cz, torch, f, block, kind, True)
    exact = _dense(cz, torch, f, block, kind, False)
    rng = float(f.max()) - float(f.min())
    d_oracle = 0.0
    for sl in _blocks(shape, block):
        want = O.fwd3d(kind, f[sl]).astype(np.float64)
        d_oracle = max(d_oracle, float(np.abs(fast[sl] - want).max()))
        np.testing.assert_array_equal(exact[sl], want)  # the exact build is the oracle
    assert d_oracle <= 2.0 ** -20 * rng, d_oracle / rng


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype,block,shape", CASES)
def test_fast_psnr_within_0p01_db_and_cr_within_1pct(dtype, block, shape, kind):
    """On fields of 54 to 192 blocks (PSNR is a whole-field figure)."""
    import torch
    from paper_1903_07761_gb300 import cz
    shape = tuple(int(1.5 * n) if n % (2 * block) == 0 and block == 32 else 2 * n for n in shape)
    shape = tuple(n - n % block for n in shape)
    f = _field(shape, dtype, seed=6)
    t = torch.from_numpy(f).cuda()
    for eps in (1e-3, 1e-4):
        out, nb = cz.compress(t, block=block, kind=kind, eps=eps, fast=True)
        n = int(nb.item())
        s = out[:n].cpu().numpy().tobytes()
        assert s[27] == cz.FLAG_FAST
        rec = cz.decompress(out, nbytes=n).cpu().numpy()
        ref = O.compress(f, block, kind, eps)
        want = O.decompress(ref)
        pg, po = O.psnr(f, rec), O.psnr(f, want)
        assert abs(pg - po) <= 0.01, (pg, po)
        assert abs(len(s) - len(ref)) <= 0.01 * len(ref)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype,block,shape", CASES)
def test_fast_strict_bound_holds(dtype, block, shape, kind):
    import torch
    from paper_1903_07761_gb300 import cz
    f = _field(shape, dtype, seed=7)
    t = torch.from_numpy(f).cuda()
    eps = 1e-3
    out, nb = cz.compress(t, block=block, kind=kind, eps=eps, fast=True, bound_mode=cz.BOUND_STRICT)
    rec = cz.decompress(out, nbytes=int(nb.item())).cpu().numpy()
    rng = float(f.max()) - float(f.min())
    ulp = np.finfo(dtype).eps * float(np.abs(f).max()) * 8
    err = float(np.abs(rec.astype(np.float64) - f.astype(np.float64)).max())
    assert err <= eps * rng + 1e-6 + ulp, (err, eps * rng)


@pytest.mark.parametrize("kind", (O.W4, O.W4LI))
def test_fast_build_refuses_w4_and_w4li(kind):
    import torch
    from paper_1903_07761_gb300 import cz
    f = torch.from_numpy(_field((32, 32, 32), np.float32)).cuda()
    with pytest.raises(cz.CzError) as e:
        cz.compress(f, block=32, kind=kind, eps=1e-3, fast=True)
    assert e.value.code == cz.ERR_ARG
