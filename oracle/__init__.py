"""CPU oracle of the CubismZ stage-1 codec -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The GPU library never links, loads or calls it,
and the two share no code.  The arithmetic lives in plain C (``czo.c`` and
``czo_real.inc``, built with ``-ffp-contract=off``); this module only builds
the shared object and marshals numpy arrays through ctypes.

What each C function follows in the paper (arXiv 1903.07761):
  * wavelets W4 / W4li / W3ai -- Sec. 2.3 "Wavelet types"; block-local "on
    the interval" transform -- Sec. 2.3 "Wavelet-based compression";
  * coefficient stream + bit-set mask -- Sec. 2.3 "Wavelet-based compression";
  * byte shuffle of coefficients and masks -- Sec. 2.3 "Lossless compression";
  * CR (with metadata) and PSNR (with the factor 2) -- Sec. 3, Eq. (1).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libczo.so")
_SRC = [os.path.join(_HERE, f) for f in ("czo.c", "czo_real.inc", "czo.h")]
_lock = threading.Lock()
_lib = None

W4, W4LI, W3AI = 0, 1, 2
F32, F64 = 0, 1
EPS_REL, EPS_ABS = 0, 1
BOUND_PAPER, BOUND_STRICT = 0, 1
FLAG_ZERO4, FLAG_ZERO8 = 2, 4  # bit zeroing of the kept details (Sec. 3, Exp. 2)
# aggregate chunks of 4 / 8 / 16 consecutive blocks (Sec. 3, Exp. 2 and 3)
FLAG_GROUP4, FLAG_GROUP8, FLAG_GROUP16 = 8, 16, 24
GROUP_MASK = 24
OK, ERR_ARG, ERR_CAPACITY, ERR_CORRUPT = 0, -1, -2, -3
HEADER_BYTES = 128


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("block", C.c_int32), ("dtype", C.c_int32), ("kind", C.c_int32),
        ("eps_mode", C.c_int32), ("stage2", C.c_int32),
        ("bound_mode", C.c_int32), ("flags", C.c_int32),
        ("eps", C.c_double), ("range", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add) into oracle/_build."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRC)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, os.path.join(_HERE, "czo.c"), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            P = C.c_void_p
            for sfx in ("f32", "f64"):
                for name in ("fwd1d", "inv1d"):
                    f = getattr(L, f"czo_{name}_{sfx}")
                    f.argtypes = [C.c_int, P, C.c_int, C.c_ssize_t]
                    f.restype = C.c_int
                for name in ("fwd3d", "inv3d"):
                    f = getattr(L, f"czo_{name}_{sfx}")
                    f.argtypes = [C.c_int, P, C.c_int]
                    f.restype = C.c_int
                f = getattr(L, f"czo_encode_block_{sfx}")
                f.argtypes = [C.c_int, C.c_int,
                              C.c_float if sfx == "f32" else C.c_double,
                              C.c_int, P, P, C.c_size_t]
                f.restype = C.c_int64
                f = getattr(L, f"czo_encode_block_z_{sfx}")
                f.argtypes = [C.c_int, C.c_int,
                              C.c_float if sfx == "f32" else C.c_double,
                              C.c_int, C.c_int, P, P, C.c_size_t]
                f.restype = C.c_int64
                f = getattr(L, f"czo_decode_block_{sfx}")
                f.argtypes = [C.c_int, C.c_int, C.c_int, P, C.c_size_t, P]
                f.restype = C.c_int
                f = getattr(L, f"czo_minmax_{sfx}")
                f.argtypes = [P, C.c_size_t, C.POINTER(C.c_double), C.POINTER(C.c_double)]
                f.restype = None
                for name in ("psnr", "linf"):
                    f = getattr(L, f"czo_{name}_{sfx}")
                    f.argtypes = [P, P, C.c_size_t]
                    f.restype = C.c_double
            L.czo_compress_bound.argtypes = [C.POINTER(Params), C.POINTER(C.c_size_t)]
            L.czo_compress.argtypes = [C.POINTER(Params), P, P, C.c_size_t, C.POINTER(C.c_size_t)]
            L.czo_decompress.argtypes = [P, C.c_size_t, P, C.c_size_t]
            L.czo_read_header.argtypes = [P, C.c_size_t, C.POINTER(Params),
                                          C.POINTER(C.c_double), C.POINTER(C.c_double),
                                          C.POINTER(C.c_double), C.POINTER(C.c_uint64)]
            L.czo_threshold.argtypes = [C.c_double, C.c_int, C.c_double]
            L.czo_threshold.restype = C.c_double
            L.czo_synthesis_norm.argtypes = [C.c_int, C.c_int]
            L.czo_synthesis_norm.restype = C.c_double
            L.czo_shuffle.argtypes = [P, C.c_size_t, C.c_int, P]
            L.czo_unshuffle.argtypes = [P, C.c_size_t, C.c_int, P]
            L.czo_rle_encode.argtypes = [P, C.c_size_t, P, C.c_size_t, C.POINTER(C.c_size_t),
                                         P, C.c_size_t, C.POINTER(C.c_size_t)]
            L.czo_rle_encode.restype = C.c_int64
            L.czo_rle_decode.argtypes = [P, C.c_size_t, P, C.c_size_t, P, C.c_size_t]
            L.czo_update_weight.argtypes = [C.c_int, C.c_int, C.c_int,
                                            C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
            _lib = L
    return _lib


def _sfx(a: np.ndarray) -> str:
    if a.dtype == np.float32:
        return "f32"
    if a.dtype == np.float64:
        return "f64"
    raise TypeError(f"unsupported dtype {a.dtype}")


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- transforms
def fwd1d(kind: int, f: np.ndarray) -> np.ndarray:
    """One level of the 1D forward transform (interleaved output)."""
    out = np.ascontiguousarray(f).copy()
    r = getattr(lib(), f"czo_fwd1d_{_sfx(out)}")(kind, _ptr(out), out.size, 1)
    assert r == OK, r
    return out


def inv1d(kind: int, f: np.ndarray) -> np.ndarray:
    out = np.ascontiguousarray(f).copy()
    r = getattr(lib(), f"czo_inv1d_{_sfx(out)}")(kind, _ptr(out), out.size, 1)
    assert r == OK, r
    return out


def fwd3d(kind: int, blk: np.ndarray) -> np.ndarray:
    """Full dyadic forward transform of one B^3 block indexed [z][y][x]."""
    out = np.ascontiguousarray(blk).copy()
    B = out.shape[0]
    assert out.shape == (B, B, B)
    r = getattr(lib(), f"czo_fwd3d_{_sfx(out)}")(kind, _ptr(out), B)
    assert r == OK, r
    return out


def inv3d(kind: int, blk: np.ndarray) -> np.ndarray:
    out = np.ascontiguousarray(blk).copy()
    B = out.shape[0]
    r = getattr(lib(), f"czo_inv3d_{_sfx(out)}")(kind, _ptr(out), B)
    assert r == OK, r
    return out


def update_weight(m: int, k: int, j: int):
    """Exact W4li update weight of detail k on coarse node j, or None."""
    n, d = C.c_int64(), C.c_int64()
    if lib().czo_update_weight(m, k, j, C.byref(n), C.byref(d)) != 0:
        return None
    return n.value, d.value


# ---------------------------------------------------------------- block codec
def encode_block(kind: int, t: float, blk: np.ndarray, stage2: bool, zbits: int = 0) -> bytes:
    blk = np.ascontiguousarray(blk)
    B = blk.shape[0]
    s = blk.dtype.itemsize
    cap = 64 * s + B ** 3 // 8 + B ** 3 * s + 4096
    out = np.zeros(cap, np.uint8)
    n = getattr(lib(), f"czo_encode_block_z_{_sfx(blk)}")(
        kind, B, t, int(stage2), int(zbits), _ptr(blk), _ptr(out), cap)
    assert n >= 0, n
    return out[:n].tobytes()


def decode_block(kind: int, B: int, dtype, chunk: bytes, stage2: bool) -> np.ndarray:
    blk = np.zeros((B, B, B), dtype)
    buf = np.frombuffer(chunk, np.uint8).copy()
    r = getattr(lib(), f"czo_decode_block_{_sfx(blk)}")(
        kind, B, int(stage2), _ptr(buf), buf.size, _ptr(blk))
    if r != OK:
        raise ValueError(f"decode_block failed: {r}")
    return blk


# ---------------------------------------------------------------- whole field
def zero_flag(zbits: int) -> int:
    return {0: 0, 4: FLAG_ZERO4, 8: FLAG_ZERO8}[int(zbits)]


def group_flag(group: int) -> int:
    return {1: 0, 4: FLAG_GROUP4, 8: FLAG_GROUP8, 16: FLAG_GROUP16}[int(group)]


def group_blocks(flags: int) -> int:
    """Blocks per chunk of a flags word: 1, 4, 8 or 16."""
    code = (int(flags) & GROUP_MASK) >> 3
    return 2 << code if code else 1


def params(shape, block, dtype, kind, eps, eps_mode=EPS_REL, stage2=True, range_=-1.0,
           bound_mode=0, zbits=0, group=1):
    nz, ny, nx = shape
    return Params(nx, ny, nz, block, F64 if np.dtype(dtype) == np.float64 else F32,
                  kind, eps_mode, int(stage2), int(bound_mode), zero_flag(zbits) | group_flag(group),
                  float(eps), float(range_))


def compress(field: np.ndarray, block: int, kind: int, eps: float,
             eps_mode: int = EPS_REL, stage2: bool = True, range_: float = -1.0,
             bound_mode: int = 0, zbits: int = 0, group: int = 1) -> bytes:
    """zbits = 4 / 8: bit zeroing Z4 / Z8 of the kept details (Sec. 3, Exp. 2).
    group = 4 / 8 / 16: aggregate chunks, each over that many consecutive
    blocks (Sec. 3, Exp. 2 and 3; stage 2 only)."""
    field = np.ascontiguousarray(field)
    p = params(field.shape, block, field.dtype, kind, eps, eps_mode, stage2, range_, bound_mode, zbits, group)
    cap = C.c_size_t()
    r = lib().czo_compress_bound(C.byref(p), C.byref(cap))
    if r != OK:
        raise ValueError(f"compress_bound failed: {r}")
    out = np.zeros(cap.value, np.uint8)
    n = C.c_size_t()
    r = lib().czo_compress(C.byref(p), _ptr(field), _ptr(out), cap.value, C.byref(n))
    if r != OK:
        raise ValueError(f"compress failed: {r}")
    return out[: n.value].tobytes()


def compress_bound(shape, block, dtype, kind=W4, stage2=True) -> int:
    p = params(shape, block, dtype, kind, 0.0, EPS_REL, stage2)
    cap = C.c_size_t()
    r = lib().czo_compress_bound(C.byref(p), C.byref(cap))
    if r != OK:
        raise ValueError(f"compress_bound failed: {r}")
    return cap.value


def read_header(stream: bytes) -> dict:
    buf = np.frombuffer(stream, np.uint8).copy()
    p = Params()
    t, mn, mx = C.c_double(), C.c_double(), C.c_double()
    tot = C.c_uint64()
    r = lib().czo_read_header(_ptr(buf), buf.size, C.byref(p), C.byref(t),
                              C.byref(mn), C.byref(mx), C.byref(tot))
    if r != OK:
        raise ValueError(f"bad header: {r}")
    return dict(nx=p.nx, ny=p.ny, nz=p.nz, block=p.block, dtype=p.dtype, kind=p.kind,
                eps_mode=p.eps_mode, stage2=p.stage2, bound_mode=p.bound_mode, flags=p.flags,
                eps=p.eps, range=p.range,
                t=t.value, min=mn.value, max=mx.value, total=tot.value)


def decompress(stream: bytes) -> np.ndarray:
    h = read_header(stream)
    dt = np.float64 if h["dtype"] == F64 else np.float32
    out = np.zeros((h["nz"], h["ny"], h["nx"]), dt)
    buf = np.frombuffer(stream, np.uint8).copy()
    r = lib().czo_decompress(_ptr(buf), buf.size, _ptr(out), out.nbytes)
    if r != OK:
        raise ValueError(f"decompress failed: {r}")
    return out


def chunk_table(stream: bytes):
    """(data_start, offsets[nchunks+1]) parsed from a stream (one chunk per
    block, or per group of blocks with a group flag)."""
    h = read_header(stream)
    B = h["block"]
    nb = (h["nx"] // B) * (h["ny"] // B) * (h["nz"] // B)
    G = group_blocks(h["flags"])
    nc = (nb + G - 1) // G
    offs = np.frombuffer(stream, np.uint64, count=nc + 1, offset=HEADER_BYTES).astype(np.int64)
    data0 = (HEADER_BYTES + 8 * (nc + 1) + 15) // 16 * 16
    return data0, offs


# ---------------------------------------------------------------- a0, metrics
def minmax(x: np.ndarray):
    x = np.ascontiguousarray(x)
    mn, mx = C.c_double(), C.c_double()
    getattr(lib(), f"czo_minmax_{_sfx(x)}")(_ptr(x), x.size, C.byref(mn), C.byref(mx))
    return mn.value, mx.value


def threshold(eps: float, eps_mode: int, range_: float) -> float:
    return lib().czo_threshold(eps, eps_mode, range_)


def psnr(R: np.ndarray, D: np.ndarray) -> float:
    R = np.ascontiguousarray(R)
    D = np.ascontiguousarray(D, dtype=R.dtype)
    return getattr(lib(), f"czo_psnr_{_sfx(R)}")(_ptr(R), _ptr(D), R.size)


def linf(R: np.ndarray, D: np.ndarray) -> float:
    R = np.ascontiguousarray(R)
    D = np.ascontiguousarray(D, dtype=R.dtype)
    return getattr(lib(), f"czo_linf_{_sfx(R)}")(_ptr(R), _ptr(D), R.size)


# ---------------------------------------------------------------- stage 2
def shuffle(b: bytes, s: int) -> bytes:
    a = np.frombuffer(b, np.uint8).copy()
    o = np.zeros_like(a)
    lib().czo_shuffle(_ptr(a), a.size, s, _ptr(o))
    return o.tobytes()


def unshuffle(b: bytes, s: int) -> bytes:
    a = np.frombuffer(b, np.uint8).copy()
    o = np.zeros_like(a)
    lib().czo_unshuffle(_ptr(a), a.size, s, _ptr(o))
    return o.tobytes()


def rle_encode(b: bytes):
    """-> (tokens as list of (literal words, zero words), literal bytes)."""
    a = np.frombuffer(b, np.uint8).copy()
    tcap = a.size // 4 + 16
    tok = np.zeros(tcap, np.uint32)
    lit = np.zeros(max(a.size, 4), np.uint8)
    nt, nl = C.c_size_t(), C.c_size_t()
    r = lib().czo_rle_encode(_ptr(a), a.size, _ptr(tok), tcap, C.byref(nt),
                             _ptr(lit), lit.size, C.byref(nl))
    assert r >= 0, r
    toks = [(int(v) & 0xFFFF, int(v) >> 16) for v in tok[: nt.value]]
    return toks, lit[: nl.value].tobytes()


def rle_decode(tokens, lits: bytes, n: int) -> bytes:
    tok = np.array([(l | (z << 16)) for l, z in tokens] or [0], np.uint32)
    li = np.frombuffer(lits, np.uint8).copy() if lits else np.zeros(1, np.uint8)
    out = np.zeros(max(n, 1), np.uint8)
    r = lib().czo_rle_decode(_ptr(tok), len(tokens), _ptr(li), len(lits), _ptr(out), n)
    if r != OK:
        raise ValueError(f"rle_decode failed: {r}")
    return out[:n].tobytes()


def synthesis_norm(kind: int, block: int) -> float:
    """C of the strict bound mode: the largest row sum of |synthesis| over
    the detail columns of one block (see czo_synthesis_norm)."""
    c = lib().czo_synthesis_norm(kind, block)
    if not c > 0:
        raise ValueError("unsupported kind / block")
    return c
