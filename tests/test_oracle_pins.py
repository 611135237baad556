"""Pins of the CPU oracle against facts that do not come from the oracle.

Every check here is fixed by mathematics or by the format definition, not by
re-typing the oracle's formulas:
  * prediction weights = Lagrange / average-interpolation weights derived
    here by solving small Vandermonde systems (Sec. 2.3 "Wavelet types":
    fourth-order interpolating and third-order average-interpolating
    wavelets; Donoho 1992);
  * lifted-update weights = the ones that give every synthesis wavelet two
    vanishing moments (lifting scheme on the interval);
  * cubic (W4, W4li) and quadratic (W3ai) fields have all-zero details;
  * 3D transform = tensor product of 1D transforms (brute-force Kronecker);
  * perfect reconstruction at eps = 0; coarse-only reconstruction at eps = inf;
  * the decoder is the linear synthesis of the kept coefficients, so the
    error is bounded by t times the synthesis norm of the detail columns;
    for one level of W4 in 1D that bound is t itself (Sec. 2.3: decimation
    errors not larger than the threshold);
  * byte shuffle = transpose of the (elements x bytes) matrix; zero-RLE
    tokens match hand-derived fixtures; lossless round trips;
  * PSNR of a known perturbation (Sec. 3, Eq. (1), with the factor 2).
"""
import ctypes as C
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KINDS = (O.W4, O.W4LI, O.W3AI)


# ------------------------------------------------------------------ helpers
def solve_exact(M, rhs):
    """Gauss-Jordan elimination over the rationals."""
    n = len(rhs)
    A = [[Fraction(v) for v in row] + [Fraction(r)] for row, r in zip(M, rhs)]
    for c in range(n):
        p = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[p] = A[p], A[c]
        A[c] = [v / A[c][c] for v in A[c]]
        for r in range(n):
            if r != c and A[r][c] != 0:
                A[r] = [a - A[r][c] * b for a, b in zip(A[r], A[c])]
    return [A[r][n] for r in range(n)]


def lagrange_weights(nodes, x):
    """Weights w with sum_j w_j p(nodes_j) = p(x) for every cubic p (exact)."""
    nodes = [Fraction(v) for v in nodes]
    x = Fraction(x)
    M = [[v ** q for v in nodes] for q in range(len(nodes))]
    return [float(w) for w in solve_exact(M, [x ** q for q in range(len(nodes))])]


def avg_interp_weights(cells, a, b):
    """Weights w with sum_j w_j avg_{cell j}(p) = avg_{[a,b]}(p), deg p <= 2.

    cells are unit cells [j, j+1].  Average of x^q over [u, v] is
    (v^{q+1} - u^{q+1}) / ((q+1)(v-u)).
    """
    def avg(u, v, q):
        u, v = Fraction(u), Fraction(v)
        return (v ** (q + 1) - u ** (q + 1)) / ((q + 1) * (v - u))
    n = len(cells)
    M = [[avg(j, j + 1, q) for j in cells] for q in range(n)]
    return [float(w) for w in solve_exact(M, [avg(a, b, q) for q in range(n)])]


def w4_predict_matrix_from_oracle(m, kind=O.W4):
    """P[k, j]: weight of coarse j in the prediction of odd sample k."""
    P = np.zeros((m, m))
    for j in range(m):
        f = np.zeros(2 * m)
        f[2 * j] = 1.0
        d = O.fwd1d(kind, f)[1::2]
        P[:, j] = -d  # d = 0 - P
    return P


def analysis_matrix(kind, n):
    W = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        W[:, j] = O.fwd1d(kind, e)
    return W


# ------------------------------------------------------------------ weights
@pytest.mark.parametrize("m", [4, 8, 16])
def test_w4_prediction_is_lagrange_on_nearest_nodes(m):
    P = w4_predict_matrix_from_oracle(m)
    for k in range(m):
        j0 = min(max(k - 1, 0), m - 4)  # nearest four coarse nodes that exist
        want = np.zeros(m)
        want[j0:j0 + 4] = lagrange_weights(range(j0, j0 + 4), k + 0.5)
        np.testing.assert_array_equal(P[k], want)


@pytest.mark.parametrize("m", [4, 8, 16])
def test_w3ai_prediction_is_average_interpolation(m):
    # constant pairs make every coarse average equal to the pair value
    for j in range(m):
        c = np.zeros(m)
        c[j] = 1.0
        f = np.repeat(c, 2)
        out = O.fwd1d(O.W3AI, f)
        np.testing.assert_array_equal(out[0::2], c)  # coarse = pair average
        d = out[1::2]
        for k in range(m):
            j0 = min(max(k - 1, 0), m - 3)
            w = avg_interp_weights(range(j0, j0 + 3), k, k + 0.5)
            want = (1.0 if j == k else 0.0) - (w[j - j0] if j0 <= j < j0 + 3 else 0.0)
            assert d[k] == want, (m, j, k, d[k], want)


@pytest.mark.parametrize("m", [4, 8, 16])
def test_w4li_synthesis_wavelets_have_two_vanishing_moments(m):
    x = np.arange(2 * m, dtype=float)
    for k in range(m):
        e = np.zeros(2 * m)
        e[2 * k + 1] = 1.0
        psi = O.inv1d(O.W4LI, e)
        assert abs(psi.sum()) < 1e-13
        assert abs((psi * x).sum()) < 1e-12
        assert abs(psi[2 * k + 1] - 1.0) < 1  # a genuine wavelet, not zero
    # the exact weights: 1/4 on both neighbours away from the boundary rows
    for k in range(4, m - 5):
        assert O.update_weight(m, k, k) == (1, 4)
        assert O.update_weight(m, k, k + 1) == (1, 4)


@pytest.mark.parametrize("m", [4, 8, 16])
def test_w4li_update_weights_solve_moment_system_exactly(m):
    """Exact rationals: sum_j U_jk M_j^p = (2k+1)^p with M from the W4 rows."""
    P = w4_predict_matrix_from_oracle(m)
    Pf = [[Fraction(round(P[k, j] * 16), 16) for j in range(m)] for k in range(m)]
    M0 = [1 + sum(Pf[k][j] for k in range(m)) for j in range(m)]
    M1 = [2 * j + sum(Pf[k][j] * (2 * k + 1) for k in range(m)) for j in range(m)]
    for k in range(m):
        tot0 = Fraction(0)
        tot1 = Fraction(0)
        nsup = 0
        for j in range(m):
            w = O.update_weight(m, k, j)
            if w is None:
                continue
            nsup += 1
            u = Fraction(*w)
            tot0 += u * M0[j]
            tot1 += u * M1[j]
        assert nsup == 2
        assert tot0 == 1 and tot1 == 2 * k + 1


def test_w4li_keeps_w4_details():
    rng = np.random.default_rng(1)
    f = rng.standard_normal(32)
    np.testing.assert_array_equal(O.fwd1d(O.W4, f)[1::2], O.fwd1d(O.W4LI, f)[1::2])


# ------------------------------------------------------------- polynomials
def poly_field(B, deg, rng, total=False):
    """Integer-coefficient polynomial of degree <= deg in each coordinate
    (total: of total degree <= deg, so that at B = 64 every sample and every
    product the transform forms stays below 2^53 and is exact in fp64)."""
    z, y, x = np.meshgrid(*(np.arange(B, dtype=float),) * 3, indexing="ij")
    f = np.zeros((B, B, B))
    for _ in range(6):
        a, b, c = rng.integers(0, deg + 1, 3)
        while total and a + b + c > deg:
            a, b, c = rng.integers(0, deg + 1, 3)
        f += rng.integers(-3, 4) * x ** a * y ** b * z ** c
    return f + rng.integers(-50, 50)


def detail_mask(B):
    Q = B // 4
    m = np.ones((B, B, B), bool)
    m[::Q, ::Q, ::Q] = False
    return m


@pytest.mark.parametrize("B", [8, 16, 32, 64])
@pytest.mark.parametrize("kind", KINDS)
def test_polynomial_reproduction_gives_zero_details(B, kind):
    rng = np.random.default_rng(B * 10 + kind)
    deg = 2 if kind == O.W3AI else 3
    f = poly_field(B, deg, rng, total=B == 64)
    c = O.fwd3d(kind, f)
    assert np.all(c[detail_mask(B)] == 0.0)
    # one degree more is not reproduced: the pin is tight
    g = f + (np.arange(B, dtype=float) ** (deg + 1))[None, None, :]
    assert np.abs(O.fwd3d(kind, g)[detail_mask(B)]).max() > 1e-3


# ------------------------------------------------------------ 3D structure
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("B", [8, 16])
def test_3d_transform_equals_kronecker_of_1d_levels(kind, B):
    rng = np.random.default_rng(7 + B + kind)
    blk = rng.standard_normal((B, B, B))
    got = O.fwd3d(kind, blk)
    ref = blk.copy()
    L = int(np.log2(B // 4))
    for lev in range(L):
        S = 1 << lev
        n = B // S
        W = analysis_matrix(kind, n)
        idx = np.arange(0, B, S)
        sub = ref[np.ix_(idx, idx, idx)]
        # x, then y, then z (array axes 2, 1, 0)
        sub = np.einsum("ij,abj->abi", W, sub)
        sub = np.einsum("ij,ajb->aib", W, sub)
        sub = np.einsum("ij,jab->iab", W, sub)
        ref[np.ix_(idx, idx, idx)] = sub
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)



# ------------------------------------------------------- reconstruction
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_eps_zero_is_near_lossless(kind, dtype):
    rng = np.random.default_rng(11)
    f = (100 + 10 * rng.standard_normal((32, 32, 64))).astype(dtype)
    s = O.compress(f, 16, kind, 0.0)
    r = O.decompress(s)
    ulp = np.finfo(dtype).eps * np.abs(f).max()
    assert np.abs(r.astype(float) - f).max() <= 64 * ulp
    # every detail kept
    data0, offs = O.chunk_table(s)
    nnz = np.frombuffer(s, np.uint32, count=1, offset=data0 + int(offs[0]))[0]
    assert nnz == 16 ** 3 - 64


def test_eps_zero_fp64_integer_field_is_exact():
    rng = np.random.default_rng(12)
    f = rng.integers(-1000, 1000, (16, 16, 16)).astype(np.float64)
    for kind in (O.W4, O.W3AI):
        r = O.decompress(O.compress(f, 16, kind, 0.0))
        np.testing.assert_array_equal(r, f)


@pytest.mark.parametrize("kind", KINDS)
def test_huge_eps_keeps_only_coarse_and_decodes_pure_prediction(kind):
    rng = np.random.default_rng(13)
    f = rng.standard_normal((16, 16, 16))
    s = O.compress(f, 16, kind, 1e300, eps_mode=O.EPS_ABS)
    data0, offs = O.chunk_table(s)
    assert np.frombuffer(s, np.uint32, count=1, offset=data0)[0] == 0
    c = O.fwd3d(kind, f)
    c[detail_mask(16)] = 0.0
    np.testing.assert_array_equal(O.decompress(s), O.inv3d(kind, c))


def test_huge_eps_on_cubic_field_is_exact():
    f = poly_field(16, 3, np.random.default_rng(14))
    s = O.compress(f, 16, O.W4, 1e300, eps_mode=O.EPS_ABS)
    np.testing.assert_array_equal(O.decompress(s), f)


@pytest.mark.parametrize("kind", KINDS)
def test_64_cubed_blocks_keep_no_details_of_a_reproduced_polynomial(kind):
    """64^3 blocks (Sec. 3, Exp. 3): four levels down to the 4^3 coarse
    cube.  A polynomial the wavelet reproduces (cubic for W4 / W4li,
    quadratic for W3ai, on dyadic integer samples) has zero details, so at
    any threshold every block's chunk holds nnz = 0 and the 64 coarse values
    alone decode the field exactly."""
    rng = np.random.default_rng(640 + kind)
    f = poly_field(64, 2 if kind == O.W3AI else 3, rng, total=True)
    f = np.concatenate([f, f[::-1].copy()], axis=0)  # two blocks along z
    s = O.compress(f, 64, kind, 1e-9, eps_mode=O.EPS_ABS, stage2=False)
    assert O.read_header(s)["block"] == 64
    data0, offs = O.chunk_table(s)
    assert len(offs) == 3
    for b in range(2):
        assert np.frombuffer(s, np.uint32, count=1, offset=data0 + int(offs[b]))[0] == 0
        assert offs[b + 1] - offs[b] == 8 + 64 * 8 + 64 ** 3 // 8  # header, coarse values, empty mask
    np.testing.assert_array_equal(O.decompress(s), f)


# ----------------------------------------------------------- threshold
def test_threshold_rule_ties_and_nan_kept():
    B = 8
    c = np.zeros((B, B, B))
    c[::2, ::2, ::2] = 7.0  # coarse
    c[0, 0, 1] = 5.0        # tie: kept
    c[0, 1, 0] = -5.0       # tie: kept
    c[1, 0, 0] = 4.9375     # just below: dropped
    c[3, 3, 3] = 6.0        # kept
    blk = O.inv3d(O.W4, c)
    assert np.array_equal(O.fwd3d(O.W4, blk), c)  # dyadic data: exact round trip
    chunk = O.encode_block(O.W4, 5.0, blk, stage2=False)
    nnz = np.frombuffer(chunk, np.uint32, count=1)[0]
    assert nnz == 3
    mask = np.frombuffer(chunk, np.uint32, count=B ** 3 // 32, offset=8 + 64 * 8)
    bits = np.unpackbits(mask.view(np.uint8), bitorder="little").reshape(B, B, B)
    want = np.zeros((B, B, B), np.uint8)
    want[0, 0, 1] = want[0, 1, 0] = want[3, 3, 3] = 1
    np.testing.assert_array_equal(bits, want)
    vals = np.frombuffer(chunk, np.float64, count=3, offset=8 + 64 * 8 + B ** 3 // 8)
    np.testing.assert_array_equal(vals, [5.0, -5.0, 6.0])  # increasing position
    # NaN detail is kept (the rule is "not below t")
    c2 = c.copy()
    blkn = O.inv3d(O.W4, c2)
    blkn[1, 1, 1] = np.nan
    chunk = O.encode_block(O.W4, 5.0, blkn, stage2=False)
    cn = O.fwd3d(O.W4, blkn)
    want_nnz = int(np.sum(~(np.abs(cn) < 5.0) & detail_mask(B)))
    assert np.frombuffer(chunk, np.uint32, count=1)[0] == want_nnz


def test_relative_threshold_uses_whole_field_range():
    rng = np.random.default_rng(15)
    f = rng.standard_normal((16, 16, 32)).astype(np.float32)
    s = O.compress(f, 16, O.W4, 1e-3)
    h = O.read_header(s)
    assert h["min"] == float(f.min()) and h["max"] == float(f.max())
    assert h["t"] == float(np.float32(1e-3 * (float(f.max()) - float(f.min()))))


# ------------------------------------------------------------ error bound
def synthesis_matrix(kind, B):
    n = B ** 3
    S = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        S[:, j] = O.inv3d(kind, e.reshape(B, B, B)).ravel()
    return S


def test_single_level_w4_error_below_threshold_1d():
    """One level in 1D: dropped details land only on their own sample."""
    rng = np.random.default_rng(16)
    f = rng.standard_normal(32)
    c = O.fwd1d(O.W4, f)
    t = 0.5
    d = c[1::2].copy()
    d[np.abs(d) < t] = 0.0
    c[1::2] = d
    err = np.abs(O.inv1d(O.W4, c) - f)
    assert err.max() < t
    assert np.all(err[0::2] == 0)


@pytest.mark.parametrize("kind", KINDS)
def test_decoder_is_linear_synthesis_and_error_is_bounded(kind):
    B = 8
    S = synthesis_matrix(kind, B)
    D = detail_mask(B).ravel()
    C = np.abs(S[:, D]).sum(axis=1).max()
    rng = np.random.default_rng(17 + kind)
    f = np.cumsum(rng.standard_normal((B, B, B)), axis=2)
    t = 0.3
    chunk = O.encode_block(kind, t, f, stage2=True)
    r = O.decode_block(kind, B, np.float64, chunk, stage2=True)
    c = O.fwd3d(kind, f).ravel()
    kept = ~(np.abs(c) < t) | ~D
    np.testing.assert_allclose(r.ravel(), S @ np.where(kept, c, 0.0), atol=1e-12)
    assert np.abs(r - f).max() <= t * C + 1e-12


# ---------------------------------------------------------------- strict bound
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("B", [8, 16])
def test_strict_norm_equals_dense_synthesis_row_sums(kind, B):
    """C from the Kronecker formula = brute force over the 3D synthesis
    columns of every detail position (Sec. 2.3's error bound, made exact)."""
    D = detail_mask(B).ravel()
    rows = np.zeros(B ** 3)
    e = np.zeros(B ** 3)
    for j in np.flatnonzero(D):
        e[j] = 1.0
        rows += np.abs(O.inv3d(kind, e.reshape(B, B, B)).ravel())
        e[j] = 0.0
    assert O.synthesis_norm(kind, B) == pytest.approx(rows.max(), rel=1e-12)


def test_strict_norm_closed_form_w3ai_b8():
    """W3ai at B = 8 has one level (m = 4).  The first sample of a line is
    f0 = A0 + d0 = (11 a0 - 4 a1 + a2)/8 + d0, so its row sum over all
    coefficients is R = 11/8 + 4/8 + 1/8 + 1 = 3 and over the coarse ones
    E = 2; every other row is smaller.  The corner sample then collects
    R^3 - E^3 = 27 - 8 = 19 from the detail columns."""
    assert O.synthesis_norm(O.W3AI, 8) == 19.0


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("B", [8, 16, 32, 64])
def test_strict_mode_keeps_error_below_nominal_threshold(kind, B):
    rng = np.random.default_rng(100 * B + kind)
    f = np.cumsum(np.cumsum(rng.standard_normal((B, 2 * B, B)), axis=2), axis=1)
    eps = 1e-2
    s = O.compress(f, B, kind, eps, O.EPS_REL, True, bound_mode=O.BOUND_STRICT)
    h = O.read_header(s)
    rng_ = float(f.max() - f.min())
    assert h["bound_mode"] == O.BOUND_STRICT
    assert h["t"] == pytest.approx(eps * rng_ / O.synthesis_norm(kind, B), rel=1e-15)
    r = O.decompress(s)
    assert np.abs(r - f).max() <= eps * rng_
    # the paper mode keeps fewer values and may exceed the nominal bound
    sp = O.compress(f, B, kind, eps, O.EPS_REL, True)
    assert len(sp) <= len(s)


# ---------------------------------------------------------------- stage 2
@pytest.mark.parametrize("s", [4, 8])
def test_shuffle_is_byte_matrix_transpose(s):
    rng = np.random.default_rng(18)
    a = rng.integers(0, 256, 37 * s, dtype=np.uint8)
    got = np.frombuffer(O.shuffle(a.tobytes(), s), np.uint8)
    np.testing.assert_array_equal(got, a.reshape(-1, s).T.ravel())
    assert O.unshuffle(got.tobytes(), s) == a.tobytes()


def _segments_to_bytes(segs):
    words = []
    for kind, *rest in segs:
        if kind == "lit":
            words += list(rest[0])
        elif kind == "zero":
            words += [0] * rest[0]
        elif kind == "litfill":
            words += [rest[1]] * rest[0]
    return np.array(words, np.uint32).tobytes()


def test_rle_tokens_match_hand_derived_fixtures():
    with open(os.path.join(GOLDEN, "rle_tokens.json")) as fh:
        cases = json.load(fh)["cases"]
    for case in cases:
        b = _segments_to_bytes(case["segments"])
        toks, lits = O.rle_encode(b)
        assert [list(t) for t in toks] == case["tokens"], case["name"]
        assert 4 * sum(t[0] for t in toks) == len(lits)
        assert O.rle_decode(toks, lits, len(b)) == b, case["name"]


@pytest.mark.parametrize("pattern", ["random", "zeros", "nozero", "sparse", "long"])
def test_rle_roundtrip_adversarial(pattern):
    rng = np.random.default_rng(sum(map(ord, pattern)))
    n = 300_000  # words
    if pattern == "random":
        a = rng.integers(0, 2 ** 32, n, dtype=np.uint32)
    elif pattern == "zeros":
        a = np.zeros(n, np.uint32)
    elif pattern == "nozero":
        a = rng.integers(1, 2 ** 32, n, dtype=np.uint32)
    elif pattern == "sparse":
        a = (rng.random(n) < 0.2).astype(np.uint32) * rng.integers(1, 2 ** 32, n, dtype=np.uint32)
    else:
        a = np.zeros(n, np.uint32)
        a[70_000:140_000] = rng.integers(1, 2 ** 32, 70_000, dtype=np.uint32)
    b = a.tobytes()
    toks, lits = O.rle_encode(b)
    assert all(0 <= l <= 65535 and 0 <= z <= 65535 for l, z in toks)
    assert O.rle_decode(toks, lits, len(b)) == b
    assert 4 * sum(z for _, z in toks) + len(lits) == len(b)
    # the literal words are exactly the words outside coded runs, in order
    coded = np.zeros(n, bool)
    pos = 0
    for l, z in toks:
        pos += l
        coded[pos:pos + z] = True
        pos += z
    np.testing.assert_array_equal(np.frombuffer(lits, np.uint32), a[~coded])
    assert np.all(a[coded] == 0)
    # every maximal zero run of >= 2 words is coded, single zero words are not
    iz = np.concatenate([[False], a == 0, [False]])
    starts = np.flatnonzero(~iz[:-1] & iz[1:])
    ends = np.flatnonzero(iz[:-1] & ~iz[1:])
    for s_, e_ in zip(starts, ends):
        assert coded[s_:e_].all() == (e_ - s_ >= 2)
        assert coded[s_:e_].any() == (e_ - s_ >= 2)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_stage2_is_lossless_over_stage1(kind, dtype):
    rough = np.cumsum(np.random.default_rng(19).standard_normal((16, 32, 32)), axis=1).astype(dtype)
    z, y, x = np.meshgrid(np.arange(16), np.arange(32), np.arange(32), indexing="ij")
    smooth = (np.sin(x / 5.0) * np.cos(y / 7.0) + 0.01 * z).astype(dtype)
    for f in (rough, smooth):
        s1 = O.compress(f, 16, kind, 1e-3, stage2=False)
        s2 = O.compress(f, 16, kind, 1e-3, stage2=True)
        np.testing.assert_array_equal(O.decompress(s1), O.decompress(s2))
        assert len(s2) <= O.compress_bound(f.shape, 16, dtype)
    assert len(s2) < len(s1)  # the smooth field has a sparse mask


# ---------------------------------------------------------------- metrics
def test_psnr_known_perturbation():
    R = np.linspace(0.0, 1.0, 1000)
    D = R + 1e-3
    assert abs(O.psnr(R, D) - 20 * np.log10(1.0 / 2e-3)) < 1e-9
    assert O.psnr(R, R) == np.inf
    assert abs(O.linf(R, D) - 1e-3) < 1e-15


def test_minmax_ignores_nan():
    x = np.array([3.0, np.nan, -2.0, 5.0])
    assert O.minmax(x) == (-2.0, 5.0)
    assert O.minmax(x.astype(np.float32)) == (-2.0, 5.0)


# ---------------------------------------------------------------- stream
def test_stream_layout_and_cr_includes_metadata():
    f = np.cumsum(np.random.default_rng(20).standard_normal((32, 32, 64)), axis=2).astype(np.float32)
    s = O.compress(f, 16, O.W3AI, 1e-2)
    h = O.read_header(s)
    assert (h["nx"], h["ny"], h["nz"], h["block"]) == (64, 32, 32, 16)
    data0, offs = O.chunk_table(s)
    assert offs[0] == 0 and np.all(np.diff(offs) > 0) and np.all(offs % 4 == 0)
    assert h["total"] == len(s) == data0 + offs[-1]
    assert len(s) <= O.compress_bound(f.shape, 16, np.float32)
    cr = f.nbytes / len(s)  # Sec. 3: CR counts metadata
    assert cr > 1


def test_corrupt_chunks_are_rejected():
    f = np.cumsum(np.random.default_rng(21).standard_normal((16, 16, 16)), axis=0)
    s = bytearray(O.compress(f, 16, O.W4, 1e-3))
    data0, offs = O.chunk_table(bytes(s))
    bad = bytearray(s)
    bad[data0:data0 + 4] = (10 ** 6).to_bytes(4, "little")  # nnz too large
    with pytest.raises(ValueError):
        O.decompress(bytes(bad))
    bad = bytearray(s)
    bad[data0 + 8:data0 + 12] = (0xFFFF).to_bytes(4, "little")  # wrong token
    with pytest.raises(ValueError):
        O.decompress(bytes(bad))
    with pytest.raises(ValueError):
        O.decompress(bytes(s[:-8]))


# ---------------------------------------------------------------- bit zeroing
def _raw_payload(chunk: bytes, B: int, dtype):
    """[nnz | 0 | coarse | mask | values] of a chunk without stage 2."""
    s = np.dtype(dtype).itemsize
    nnz = int(np.frombuffer(chunk[:4], np.uint32)[0])
    p = chunk[8:]
    coarse = np.frombuffer(p[:64 * s], dtype)
    mask = np.frombuffer(p[64 * s:64 * s + B ** 3 // 8], np.uint8)
    vals = np.frombuffer(p[64 * s + B ** 3 // 8:64 * s + B ** 3 // 8 + nnz * s], dtype)
    return nnz, coarse, mask, vals


@pytest.mark.parametrize("dtype,B", [(np.float32, 32), (np.float32, 8), (np.float64, 16)])
@pytest.mark.parametrize("kind", [O.W4, O.W4LI, O.W3AI])
def test_bit_zeroing_clears_the_low_bits_of_the_kept_details_only(dtype, B, kind):
    """Sec. 3, Exp. 2 (Z4 / Z8): the zbits least significant bits of every
    kept detail coefficient are zeroed; which details are kept, the mask and
    the coarse values do not change.  Checked against numpy bit masks of the
    unzeroed chunk's values."""
    rng = np.random.default_rng(kind * 10 + B)
    blk = (rng.standard_normal((B, B, B)) * rng.uniform(0.1, 10, (B, B, B))).astype(dtype)
    base = O.encode_block(kind, 0.5, blk, stage2=False)
    n0, c0, m0, v0 = _raw_payload(base, B, dtype)
    assert n0 > 0
    ut = np.uint32 if np.dtype(dtype).itemsize == 4 else np.uint64
    for zbits in (4, 8):
        ch = O.encode_block(kind, 0.5, blk, stage2=False, zbits=zbits)
        n, c, m, v = _raw_payload(ch, B, dtype)
        assert n == n0
        np.testing.assert_array_equal(m, m0)
        np.testing.assert_array_equal(c.view(ut), c0.view(ut))
        want = v0.view(ut) & ~ut((1 << zbits) - 1)
        np.testing.assert_array_equal(v.view(ut), want)
        assert np.any(v.view(ut) != v0.view(ut))
        # the same block through stage 2 decodes to the same values
        ch2 = O.encode_block(kind, 0.5, blk, stage2=True, zbits=zbits)
        np.testing.assert_array_equal(O.decode_block(kind, B, dtype, ch2, True).view(ut),
                                      O.decode_block(kind, B, dtype, ch, False).view(ut))


def test_bit_zeroing_flags_and_header():
    f = np.random.default_rng(3).standard_normal((32, 32, 64)).astype(np.float32)
    for zbits, flag in ((0, 0), (4, O.FLAG_ZERO4), (8, O.FLAG_ZERO8)):
        s = O.compress(f, 16, O.W3AI, 1e-2, zbits=zbits)
        assert s[27] == flag and O.read_header(s)["flags"] == flag
    p = O.params(f.shape, 16, f.dtype, O.W3AI, 1e-2)
    cap = C.c_size_t()
    for flags, bound in ((O.FLAG_ZERO4 | O.FLAG_ZERO8, O.BOUND_PAPER), (O.FLAG_ZERO8, O.BOUND_STRICT)):
        p.flags, p.bound_mode = flags, bound
        assert O.lib().czo_compress_bound(C.byref(p), C.byref(cap)) == O.ERR_ARG


def test_z8_shrinks_the_stage2_stream_of_a_smooth_field():
    """Zeroing the low byte of every kept FP32 detail empties one shuffled
    byte plane of the values, which the zero-run coder removes; the decoded
    field moves by at most 2^8 ulp per kept coefficient."""
    from paper_1903_07761_gb300 import inputs
    f = inputs.config0(seed=0)
    s0 = O.compress(f, 32, O.W3AI, 1e-3)
    s8 = O.compress(f, 32, O.W3AI, 1e-3, zbits=8)
    assert len(s8) < len(s0)
    assert abs(O.psnr(f, O.decompress(s8)) - O.psnr(f, O.decompress(s0))) < 0.1


@pytest.mark.parametrize("dtype,B", [(np.float64, 32), (np.float32, 64)])
def test_payloads_longer_than_a_token_field_split_as_defined(dtype, B):
    """FP64 32^3 and FP32 64^3 payloads can exceed 65535 words (every
    detail kept, eps = 0, on noise: no zero words).  A chunk then starts with
    (65535, 0) tokens, one per full token field of literals, and the rest;
    the literal words are the whole shuffled payload, and the stream decodes
    to the exact transform's inverse."""
    rng = np.random.default_rng(B)
    f = rng.standard_normal((B, B, B)).astype(dtype)
    s = O.compress(f, B, O.W4, 0.0)
    d0, offs = O.chunk_table(s)
    ch = s[d0 + int(offs[0]):d0 + int(offs[1])]
    nnz, ntok = np.frombuffer(ch, np.uint32, count=2)
    es = np.dtype(dtype).itemsize
    W = (64 * es + B ** 3 // 8 + int(nnz) * es) // 4
    assert nnz == B ** 3 - 64 and W > 65535
    toks = np.frombuffer(ch, np.uint32, count=int(ntok), offset=8)
    lit, zr = toks & 0xFFFF, toks >> 16
    full = W // 65535 if W % 65535 else W // 65535 - 1
    assert list(toks[:full]) == [65535] * full  # (65535, 0) while more than 65535 literals remain
    assert int(lit.sum()) + int(zr.sum()) == W
    assert len(ch) == 8 + 4 * int(ntok) + 4 * int(lit.sum())
    np.testing.assert_array_equal(O.decompress(s), O.inv3d(O.W4, O.fwd3d(O.W4, f)).astype(dtype))
