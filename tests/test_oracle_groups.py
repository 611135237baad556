"""Pins of the oracle's aggregate chunks (Sec. 3, Exp. 2 and 3: the stage-1
output of several consecutive blocks is concatenated and the lossless
substage codes the concatenation as one buffer).

Nothing here re-uses the oracle's group code to check itself:
  * every group chunk is taken apart by code written here (a plain token
    walk and a numpy byte transpose), and the bytes it yields must equal the
    concatenated raw payloads of the same blocks as they appear in the
    stream without stage 2 (one chunk per block, no shuffle, no coding), and
    its nnz words the per-block chunks' nnz words;
  * the coding is lossless, so the decoded field equals the one of the
    per-block stream bit for bit;
  * the offset table has one entry per group (ceil(nblocks / G) + 1), the
    header keeps the block count and carries the group code.
"""
import numpy as np
import pytest

import oracle as O


def _field(shape, dtype, seed, noise=1e-3):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64) for n in shape), indexing="ij")
    f = 40 + 15 * np.sin(x / 5.3 + rng.random()) * np.cos(y / 4.1) + 4 * np.sin(z / 2.9)
    f += 6 * np.exp(-((x - shape[2] / 3) ** 2 + (z - shape[0] / 2) ** 2) / 20.0)
    f += noise * rng.standard_normal(shape)
    return f.astype(dtype)


def _words(b: bytes, off: int, n: int):
    return np.frombuffer(b, np.uint32, count=n, offset=off)


def _raw_payloads(stream_plain: bytes):
    """(nnz, payload bytes) of every block of a stream without stage 2:
    chunk = [nnz | 0 | payload]."""
    data0, offs = O.chunk_table(stream_plain)
    out = []
    for c in range(len(offs) - 1):
        ch = stream_plain[data0 + offs[c]: data0 + offs[c + 1]]
        nnz, zero = _words(ch, 0, 2)
        assert zero == 0
        out.append((int(nnz), ch[8:]))
    return out


def _untoken(tokens, lits: bytes, nwords: int) -> bytes:
    """Plain walk over (literal words, zero words) tokens."""
    out, li = [], 0
    for t in tokens:
        n, z = int(t) & 0xFFFF, int(t) >> 16
        out.append(lits[4 * li: 4 * (li + n)])
        li += n
        out.append(bytes(4 * z))
    b = b"".join(out)
    assert len(b) == 4 * nwords and 4 * li == len(lits)
    return b


def _unshuffle(b: bytes, s: int) -> bytes:
    """Byte plane q holds byte q of every s-byte element: a transpose."""
    a = np.frombuffer(b, np.uint8)
    return a.reshape(s, len(a) // s).T.reshape(-1).tobytes()


CASES = [
    # (shape, block, dtype, group): ragged last groups (12 blocks of 32^3,
    # 60 of 16^3, 192 of 8^3) and full ones
    ((64, 64, 96), 32, np.float32, 8),
    ((64, 64, 96), 32, np.float32, 16),
    ((48, 80, 64), 16, np.float32, 8),
    ((48, 80, 64), 16, np.float64, 4),
    ((32, 48, 64), 8, np.float32, 16),
    ((32, 48, 64), 8, np.float64, 4),
]


@pytest.mark.parametrize("shape,block,dtype,group", CASES)
@pytest.mark.parametrize("kind", (O.W4, O.W4LI, O.W3AI))
def test_group_chunk_is_the_coded_concatenation(shape, block, dtype, group, kind):
    f = _field(shape, dtype, seed=block + group + kind)
    s = np.dtype(dtype).itemsize
    plain = _raw_payloads(O.compress(f, block, kind, 1e-3, stage2=False))
    sg = O.compress(f, block, kind, 1e-3, group=group)
    h = O.read_header(sg)
    nb = len(plain)
    assert O.group_blocks(h["flags"]) == group
    assert int.from_bytes(sg[28:32], "little") == nb
    data0, offs = O.chunk_table(sg)
    ng = -(-nb // group)
    assert len(offs) == ng + 1 and offs[0] == 0
    assert data0 == (O.HEADER_BYTES + 8 * (ng + 1) + 15) // 16 * 16
    assert data0 + offs[-1] == len(sg)
    for c in range(ng):
        blocks = plain[c * group:(c + 1) * group]
        g = len(blocks)
        ch = sg[data0 + offs[c]: data0 + offs[c + 1]]
        head = _words(ch, 0, g + 1)
        assert [int(v) for v in head[:g]] == [nnz for nnz, _ in blocks]
        ntok = int(head[g])
        toks = _words(ch, 4 * (g + 1), ntok)
        lits = ch[4 * (g + 1) + 4 * ntok:]
        concat = b"".join(p for _, p in blocks)
        assert len(concat) % s == 0
        assert _unshuffle(_untoken(toks, lits, len(concat) // 4), s) == concat


@pytest.mark.parametrize("shape,block,dtype,group", CASES)
def test_group_stream_decodes_like_the_per_block_stream(shape, block, dtype, group):
    f = _field(shape, dtype, seed=7 * block + group)
    for eps in (0.0, 1e-4, 1e-2):
        want = O.decompress(O.compress(f, block, O.W3AI, eps))
        got = O.decompress(O.compress(f, block, O.W3AI, eps, group=group))
        assert got.tobytes() == want.tobytes()


def test_every_detail_kept_in_a_group():
    """eps = 0 on noise: group payloads of 16 blocks x 17 KiB (16^3 FP32),
    literal runs beyond a token's 65535 words are split."""
    f = np.random.default_rng(3).standard_normal((16, 32, 128)).astype(np.float32)
    sg = O.compress(f, 16, O.W4, 0.0, group=16)
    data0, offs = O.chunk_table(sg)
    assert len(offs) == 2
    ch = sg[data0:]
    ntok = int(_words(ch, 64, 1)[0])
    assert ntok >= 2  # 16 x 4352 words of literals: at least one split
    assert O.decompress(sg).tobytes() == O.decompress(O.compress(f, 16, O.W4, 0.0)).tobytes()


def test_group_needs_stage2_and_flags_decode():
    f = _field((32, 32, 32), np.float32, seed=1)
    with pytest.raises(ValueError):
        O.compress(f, 16, O.W3AI, 1e-3, stage2=False, group=4)
    assert [O.group_blocks(v) for v in (0, 8, 16, 24, 2 | 16)] == [1, 4, 8, 16, 8]


def test_corrupt_group_chunk_is_refused():
    f = _field((32, 32, 64), np.float32, seed=2)
    sg = bytearray(O.compress(f, 16, O.W3AI, 1e-3, group=4))
    data0, offs = O.chunk_table(bytes(sg))
    # first block's nnz beyond the detail count of a block
    sg[data0:data0 + 4] = (16 ** 3).to_bytes(4, "little")
    with pytest.raises(ValueError):
        O.decompress(bytes(sg))
