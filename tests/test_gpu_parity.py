"""GPU path vs the CPU oracle, through the C ABI.

The GPU kernels evaluate every wavelet step in the oracle's operation order
with explicitly rounded (never fused) arithmetic, so streams, masks and
decoded fields must be bit-identical to the oracle's.  Floating point decides
which details are kept (a threshold compare), so both sides take that
decision in the field's own precision.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import describe_diff, gpu_compress, gpu_decompress

pytestmark = pytest.mark.gpu

KINDS = (O.W4, O.W4LI, O.W3AI)
# (dtype, block, shape) with ragged block grids
CASES = [
    (np.float32, 32, (32, 64, 96)),
    (np.float32, 16, (16, 48, 32)),
    (np.float32, 8, (8, 24, 40)),
    (np.float64, 16, (32, 16, 48)),
    (np.float64, 8, (24, 8, 16)),
    (np.float64, 32, (32, 64, 96)),  # 256 KiB blocks: the slab kernels
    (np.float32, 64, (64, 64, 128)),  # 1 MiB blocks: the slab kernels, four levels
]


def smooth_field(shape, dtype, seed):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64) for n in shape), indexing="ij")
    f = 50 + 20 * np.sin(x / 7.3 + rng.random()) * np.cos(y / 5.1) + 3 * np.sin(z / 3.7)
    f += 5 * np.exp(-((x - shape[2] / 2) ** 2 + (y - shape[1] / 3) ** 2) / 30.0)
    f += 1e-3 * rng.standard_normal(shape)
    return f.astype(dtype)


def test_config0_small_case_stream_is_bit_identical():
    """128^3 FP32 Gaussian bubbles, 64 blocks of 32^3, W4, eps = 1e-3 * range."""
    from paper_1903_07761_gb300 import inputs
    f = inputs.config0(seed=0)
    ref = O.compress(f, 32, O.W4, 1e-3)
    got = gpu_compress(f, 32, O.W4, 1e-3)
    assert got == ref, describe_diff(got, ref)
    rec = gpu_decompress(got)
    np.testing.assert_array_equal(rec.view(np.uint32), O.decompress(ref).view(np.uint32))
    # the decoded fields are identical, hence so are PSNR and CR (51.26 dB, 144.6x)
    assert abs(O.psnr(f, rec) - O.psnr(f, O.decompress(ref))) < 0.01
    assert 45 < O.psnr(f, rec) < 60


@pytest.mark.parametrize("stage2", [True, False])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype,block,shape", CASES)
def test_stream_and_decode_bit_identical(dtype, block, shape, kind, stage2):
    f = smooth_field(shape, dtype, seed=block + kind)
    for eps in (1e-3, 1e-2):
        ref = O.compress(f, block, kind, eps, stage2=stage2)
        got = gpu_compress(f, block, kind, eps, stage2=stage2)
        assert got == ref, f"eps={eps}: " + describe_diff(got, ref)
        rec = gpu_decompress(got)
        want = O.decompress(ref)
        np.testing.assert_array_equal(rec.view(np.uint8), want.view(np.uint8))


@pytest.mark.parametrize("zbits", [4, 8])
@pytest.mark.parametrize("stage2", [True, False])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype,block,shape", [CASES[0], CASES[3], CASES[5]])
def test_bit_zeroing_streams_bit_identical(dtype, block, shape, kind, stage2, zbits):
    """Bit zeroing Z4 / Z8 (Sec. 3, Exp. 2): the kept details' low bits are
    cleared on the GPU exactly as in the oracle."""
    f = smooth_field(shape, dtype, seed=31 + kind)
    ref = O.compress(f, block, kind, 1e-3, stage2=stage2, zbits=zbits)
    got = gpu_compress(f, block, kind, 1e-3, stage2=stage2, zbits=zbits)
    assert got == ref, describe_diff(got, ref)
    np.testing.assert_array_equal(gpu_decompress(got).view(np.uint8), O.decompress(ref).view(np.uint8))


@pytest.mark.parametrize("stage2", [True, False])
@pytest.mark.parametrize("dtype,block,shape", [
    (np.float32, 32, (64, 160, 544)),  # 17 x 5 x 2 = 170 blocks: more than one per stage CTA
    (np.float64, 16, (64, 96, 400)),   # 25 x 6 x 4 = 600 blocks
    (np.float64, 32, (64, 160, 1024)),  # 32 x 5 x 2 = 320 blocks of 32^3 (more than one per slab CTA)
])
def test_non_cubic_grid_with_several_blocks_per_cta(dtype, block, shape, stage2):
    """The persistent kernels walk their blocks in steps of the grid size
    over a non-cubic block grid (carries in x and y); every block's tile and
    output tile must land at its own coordinates."""
    f = smooth_field(shape, dtype, seed=5)
    ref = O.compress(f, block, O.W3AI, 1e-3, stage2=stage2)
    got = gpu_compress(f, block, O.W3AI, 1e-3, stage2=stage2)
    assert got == ref, describe_diff(got, ref)
    rec = gpu_decompress(got)
    np.testing.assert_array_equal(rec.view(np.uint8), O.decompress(ref).view(np.uint8))


@pytest.mark.parametrize("dtype,block", [(np.float64, 16), (np.float32, 16), (np.float64, 32)])
def test_payload_exactly_at_the_stage2_shared_capacity(dtype, block):
    """One block whose payload is exactly 16 KiB (the stage-2 kernels'
    shared-memory capacity) and has no zero-word runs, so its finished chunk
    is 12 bytes longer than the payload: it must be encoded once, by the
    small-payload launch.  The block is built from chosen coefficients: the
    synthesis of exactly nnz details of magnitude in [1, 2] (all kept) plus
    random coarse values, every other coefficient zero (rounding noise far
    below the threshold)."""
    es = np.dtype(dtype).itemsize
    nnz = (16384 - 64 * es - block ** 3 // 8) // es
    rng = np.random.default_rng(99)
    Q = block // 4
    coarse = np.zeros((block,) * 3, bool)
    coarse[::Q, ::Q, ::Q] = True
    det = np.flatnonzero(~coarse.ravel())
    c = np.zeros(block ** 3)
    pick = rng.choice(det, nnz, replace=False)
    c[pick] = rng.uniform(1, 2, nnz) * rng.choice([-1.0, 1.0], nnz)
    c[coarse.ravel()] = rng.uniform(-4, 4, 64)
    blk = O.inv3d(O.W3AI, c.reshape((block,) * 3))
    f = np.concatenate([blk, blk[::-1].copy()], axis=2).astype(dtype)  # two blocks along x
    for stage2 in (True, False):
        ref = O.compress(f, block, O.W3AI, 1e-3, eps_mode=O.EPS_ABS, stage2=stage2)
        got = gpu_compress(f, block, O.W3AI, 1e-3, eps_mode=O.EPS_ABS, stage2=stage2)
        assert got == ref, describe_diff(got, ref)
        np.testing.assert_array_equal(gpu_decompress(got).view(np.uint8), O.decompress(ref).view(np.uint8))
    d0, offs = O.chunk_table(ref)
    assert int(np.frombuffer(ref[d0:d0 + 4], np.uint32)[0]) == nnz  # the first block is at the capacity


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype,block,shape", CASES)
def test_strict_bound_mode(dtype, block, shape, kind):
    """Strict bound: threshold eps * range / C; the stream equals the oracle's
    and the decoded error stays below eps * range."""
    f = smooth_field(shape, dtype, seed=11 + kind)
    eps = 1e-2
    ref = O.compress(f, block, kind, eps, bound_mode=O.BOUND_STRICT)
    got = gpu_compress(f, block, kind, eps, bound_mode=O.BOUND_STRICT)
    assert got == ref, describe_diff(got, ref)
    rec = gpu_decompress(got)
    np.testing.assert_array_equal(rec.view(np.uint8), O.decompress(ref).view(np.uint8))
    rng_ = float(f.max()) - float(f.min())
    ulp = np.finfo(dtype).eps * float(np.abs(f).max()) * 8  # rounding of the reconstruction itself
    assert np.abs(rec.astype(np.float64) - f.astype(np.float64)).max() <= eps * rng_ + ulp


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype,block,shape", CASES)
def test_eps_zero_and_huge(dtype, block, shape, kind):
    f = smooth_field(shape, dtype, seed=7)
    for eps, mode in ((0.0, O.EPS_REL), (1e300, O.EPS_ABS)):
        ref = O.compress(f, block, kind, eps, eps_mode=mode)
        got = gpu_compress(f, block, kind, eps, eps_mode=mode)
        assert got == ref, f"eps={eps}: " + describe_diff(got, ref)
        np.testing.assert_array_equal(gpu_decompress(got).view(np.uint8),
                                      O.decompress(ref).view(np.uint8))


@pytest.mark.parametrize("dtype,block,shape", CASES)
def test_random_noise_and_supplied_range(dtype, block, shape):
    rng = np.random.default_rng(3)
    f = rng.standard_normal(shape).astype(dtype)
    for kind in KINDS:
        ref = O.compress(f, block, kind, 0.05, range_=7.5)
        got = gpu_compress(f, block, kind, 0.05, range_=7.5)
        assert got == ref, describe_diff(got, ref)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype,block,shape", CASES)
def test_dense_coefficients_match_oracle_per_block(dtype, block, shape, kind):
    import torch
    from paper_1903_07761_gb300 import cz
    f = smooth_field(shape, dtype, seed=11)
    ft = torch.from_numpy(f).cuda()
    coef = torch.empty_like(ft)
    p = cz.params_for(shape, dtype == np.float64, block, kind, 0.0)
    assert cz.cz_forward_dense(p, ft.data_ptr(), coef.data_ptr(), 0) == cz.OK
    back = torch.empty_like(ft)
    assert cz.cz_inverse_dense(p, coef.data_ptr(), back.data_ptr(), 0) == cz.OK
    torch.cuda.synchronize()
    c = coef.cpu().numpy()
    b = back.cpu().numpy()
    nz, ny, nx = shape
    for bz in range(nz // block):
        for by in range(ny // block):
            for bx in range(nx // block):
                sl = (slice(bz * block, (bz + 1) * block), slice(by * block, (by + 1) * block),
                      slice(bx * block, (bx + 1) * block))
                want = O.fwd3d(kind, f[sl])
                np.testing.assert_array_equal(c[sl].view(np.uint8), want.view(np.uint8))
                np.testing.assert_array_equal(b[sl].view(np.uint8),
                                              O.inv3d(kind, want).view(np.uint8))


def test_single_block_and_all_constant_field():
    for dtype, block in ((np.float32, 32), (np.float64, 16), (np.float32, 8), (np.float64, 32), (np.float32, 64)):
        f = np.full((block,) * 3, 3.25, dtype)
        for kind in KINDS:
            ref = O.compress(f, block, kind, 1e-3)
            got = gpu_compress(f, block, kind, 1e-3)
            assert got == ref, describe_diff(got, ref)
            np.testing.assert_array_equal(gpu_decompress(got), f)


def test_nan_values_are_kept_like_the_oracle():
    f = smooth_field((32, 32, 32), np.float32, seed=5)
    f[3, 4, 5] = np.nan
    f[20, 1, 30] = np.nan
    # NaN payload bits may differ between CPU and GPU arithmetic, and with
    # stage 2 they can change zero-word runs; without stage 2 the layout is
    # fixed by which details are kept, which must agree.
    ref = O.compress(f, 32, O.W3AI, 1e-3, stage2=False)
    got = gpu_compress(f, 32, O.W3AI, 1e-3, stage2=False)
    assert len(got) == len(ref)
    hg, hr = O.read_header(got), O.read_header(ref)
    assert hg["min"] == hr["min"] and hg["max"] == hr["max"] and hg["t"] == hr["t"]
    _, og = O.chunk_table(got)
    _, orf = O.chunk_table(ref)
    np.testing.assert_array_equal(og, orf)
    rec = gpu_decompress(got)
    want = O.decompress(ref)
    np.testing.assert_array_equal(np.isnan(rec), np.isnan(want))
    ok = ~np.isnan(want)
    np.testing.assert_array_equal(rec[ok].view(np.uint32), want[ok].view(np.uint32))


@pytest.mark.parametrize("stage2", [True, False])
@pytest.mark.parametrize("kind", KINDS)
def test_fp64_32_payloads_beyond_one_token_field(kind, stage2):
    """FP64 32^3 blocks with every detail kept (eps = 0): a payload of
    66,560 words.  Without zero words the literal run is longer than a
    token's 16-bit field and splits into (65535, 0) and the rest; on a
    constant field (every detail exactly 0, all kept) the zero-word runs of
    the shuffled payload are long.  Both go through the global-scratch
    stage-2 coder and decoder."""
    rng = np.random.default_rng(17 + kind)
    noisy = rng.standard_normal((32, 32, 64))
    const = np.full((32, 32, 32), -1.5)
    for f in (noisy, const):
        ref = O.compress(f, 32, kind, 0.0, stage2=stage2)
        got = gpu_compress(f, 32, kind, 0.0, stage2=stage2)
        assert got == ref, describe_diff(got, ref)
        np.testing.assert_array_equal(gpu_decompress(got).view(np.uint8), O.decompress(ref).view(np.uint8))
    if stage2:
        d0, offs = O.chunk_table(O.compress(noisy, 32, kind, 0.0))
        toks = np.frombuffer(O.compress(noisy, 32, kind, 0.0)[d0 + 8:d0 + 16], np.uint32)
        assert toks[0] == 65535  # the first token of a split literal run
