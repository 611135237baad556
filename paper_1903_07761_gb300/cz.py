"""Python binding of the C ABI in include/cz.h (argument marshalling only).

Every compute step runs in the CUDA kernels of ``libcz.so``; this module
loads the library (building it first if it is missing or stale), fills the
``cz_params`` struct, and passes device pointers and the current torch CUDA
stream through ctypes.  There is no CPU fallback: if the library cannot be
loaded, importing the functions raises.

The functions named ``cz_*`` mirror the ABI one to one.  ``compress`` /
``decompress`` are thin conveniences over them for torch CUDA tensors.
"""
from __future__ import annotations

import ctypes as C
import threading

from . import _build

W4, W4LI, W3AI = 0, 1, 2
F32, F64 = 0, 1
EPS_REL, EPS_ABS = 0, 1
BOUND_PAPER, BOUND_STRICT = 0, 1
FLAG_FAST = 1
FLAG_ZERO4, FLAG_ZERO8 = 2, 4  # bit zeroing Z4 / Z8 of the kept details
FLAG_GROUP4, FLAG_GROUP8, FLAG_GROUP16 = 8, 16, 24  # aggregate chunks of 4 / 8 / 16 blocks
GROUP_FLAGS = {1: 0, 4: FLAG_GROUP4, 8: FLAG_GROUP8, 16: FLAG_GROUP16}
OK, ERR_ARG, ERR_CAPACITY, ERR_CORRUPT, ERR_TIMEOUT, ERR_CUDA, ERR_BUDGET = 0, -1, -2, -3, -4, -5, -6
HEADER_BYTES = 128
NOALLOC_WS_BYTES = 64 << 20  # CZ_NOALLOC_WS_BYTES
KINDS = {"w4": W4, "w4li": W4LI, "w3ai": W3AI}


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("block", C.c_int32), ("dtype", C.c_int32), ("kind", C.c_int32),
        ("eps_mode", C.c_int32), ("stage2", C.c_int32),
        ("bound_mode", C.c_int32), ("flags", C.c_int32),
        ("eps", C.c_double), ("range", C.c_double),
    ]


OP_COMPRESS, OP_DECOMPRESS = 0, 1
REQ_QUEUED, REQ_RUNNING, REQ_DONE = 0, 1, 2


class Request(C.Structure):
    _fields_ = [
        ("op", C.c_int32), ("reserved", C.c_int32), ("params", Params),
        ("d_in", C.c_void_p), ("in_bytes", C.c_size_t), ("h_header", C.c_ubyte * HEADER_BYTES),
        ("d_out", C.c_void_p), ("out_cap", C.c_size_t), ("d_out_bytes", C.c_void_p),
    ]


class CzError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {cz_strerror(code)} ({code})" if what else cz_strerror(code))


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded libcz.so (built in-tree on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            P = C.c_void_p
            PP = C.POINTER(Params)
            L.cz_compress_bound.argtypes = [PP, C.POINTER(C.c_size_t)]
            L.cz_workspace_size.argtypes = [PP, C.POINTER(C.c_size_t)]
            L.cz_compress.argtypes = [PP, P, P, C.c_size_t, P, P, C.c_size_t, P]
            L.cz_decompress.argtypes = [P, C.c_size_t, P, P, C.c_size_t, P, C.c_size_t, P]
            L.cz_decompress_blocks.argtypes = [P, C.c_size_t, P, P, C.c_int, P, C.c_size_t, P, C.c_size_t, P]
            L.cz_decompress_blocks_workspace_size.argtypes = [PP, C.c_int, C.POINTER(C.c_size_t)]
            L.cz_compress_noalloc.argtypes = [PP, P, P, C.c_size_t, P, P]
            L.cz_noalloc_status.argtypes = [P]
            L.cz_stream_concat.argtypes = [C.c_int, C.POINTER(P), C.POINTER(C.c_size_t), P, C.c_size_t,
                                           C.POINTER(C.c_size_t)]
            L.cz_server_create.argtypes = [C.c_size_t, C.c_int, C.POINTER(P)]
            L.cz_server_submit.argtypes = [P, C.POINTER(Request), C.POINTER(C.c_uint64)]
            L.cz_server_poll.argtypes = [P, C.c_uint64, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                         C.POINTER(C.c_double)]
            L.cz_server_wait.argtypes = [P, C.c_uint64, C.POINTER(C.c_int), C.POINTER(C.c_double)]
            L.cz_server_destroy.argtypes = [P]
            L.cz_batch_workspace_size.argtypes = [C.c_int, PP, C.POINTER(C.c_size_t)]
            L.cz_compress_batch.argtypes = [C.c_int, PP, C.POINTER(P), C.POINTER(P),
                                            C.POINTER(C.c_size_t), P, P, C.c_size_t, P]
            L.cz_batch_tune.argtypes = [C.c_int, PP, C.POINTER(P), C.POINTER(P),
                                        C.POINTER(C.c_size_t), P, P, C.c_size_t, P, C.c_int]
            L.cz_read_header.argtypes = [P, C.c_size_t, PP, C.POINTER(C.c_double)]
            L.cz_status.argtypes = [P, P]
            L.cz_strerror.argtypes = [C.c_int]
            L.cz_strerror.restype = C.c_char_p
            L.cz_forward_dense.argtypes = [PP, P, P, P]
            L.cz_inverse_dense.argtypes = [PP, P, P, P]
            L.cz_batch_knobs_export.argtypes = [P, C.c_size_t, C.POINTER(C.c_size_t)]
            L.cz_batch_knobs_import.argtypes = [C.c_char_p]
            L.cz_aos_workspace_size.argtypes = [C.c_int, PP, C.POINTER(C.c_size_t)]
            L.cz_compress_aos.argtypes = [C.c_int, PP, P, C.c_int, P, C.POINTER(P), C.POINTER(C.c_size_t), P, P,
                                          C.c_size_t, P]
            L.cz_cache_create.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(P)]
            L.cz_cache_destroy.argtypes = [P]
            L.cz_cache_destroy.restype = None
            L.cz_cache_fetch.argtypes = [P, P, C.c_size_t, P, P, C.c_int, P, C.c_size_t, P, C.c_size_t, P,
                                         C.POINTER(C.c_int)]
            L.cz_cache_clear.argtypes = [P]
            L.cz_cache_stats.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
            for f in (L.cz_compress_bound, L.cz_workspace_size, L.cz_compress, L.cz_decompress, L.cz_decompress_blocks,
                      L.cz_decompress_blocks_workspace_size, L.cz_cache_create, L.cz_cache_fetch, L.cz_cache_clear,
                      L.cz_cache_stats, L.cz_aos_workspace_size, L.cz_compress_aos, L.cz_batch_knobs_export,
                      L.cz_batch_knobs_import,
                      L.cz_compress_noalloc, L.cz_noalloc_status, L.cz_batch_workspace_size, L.cz_compress_batch,
                      L.cz_batch_tune, L.cz_stream_concat, L.cz_server_create, L.cz_server_submit, L.cz_server_poll,
                      L.cz_server_wait, L.cz_server_destroy, L.cz_read_header, L.cz_status, L.cz_forward_dense, L.cz_inverse_dense):
                f.restype = C.c_int
            _lib = L
    return _lib


# ------------------------------------------------------------------ raw ABI
def cz_compress_bound(p: Params) -> int:
    n = C.c_size_t()
    r = lib().cz_compress_bound(C.byref(p), C.byref(n))
    if r != OK:
        raise CzError(r, "cz_compress_bound")
    return n.value


def cz_workspace_size(p: Params) -> int:
    n = C.c_size_t()
    r = lib().cz_workspace_size(C.byref(p), C.byref(n))
    if r != OK:
        raise CzError(r, "cz_workspace_size")
    return n.value


def cz_compress(p: Params, d_field: int, d_out: int, out_cap: int, d_out_bytes: int,
                d_ws: int, ws_bytes: int, stream: int) -> int:
    return lib().cz_compress(C.byref(p), d_field, d_out, out_cap, d_out_bytes or None,
                             d_ws, ws_bytes, stream or None)


def cz_compress_noalloc(p: Params, d_field: int, d_out: int, out_cap: int, d_out_bytes: int,
                        stream: int) -> int:
    """cz_compress with the library's own fixed workspace (no allocation)."""
    return lib().cz_compress_noalloc(C.byref(p), d_field, d_out, out_cap, d_out_bytes or None,
                                     stream or None)


def cz_noalloc_status(stream: int) -> int:
    """Device status word of the last cz_compress_noalloc call (synchronises)."""
    return lib().cz_noalloc_status(stream or None)


class BatchArgs:
    """ctypes arrays of one batched call (kept alive by the caller)."""

    def __init__(self, params, d_fields, d_outs, out_caps):
        n = len(params)
        self.n = n
        self.params = (Params * n)(*params)
        self.fields = (C.c_void_p * n)(*d_fields)
        self.outs = (C.c_void_p * n)(*d_outs)
        self.caps = (C.c_size_t * n)(*out_caps)


def cz_batch_workspace_size(params) -> int:
    n = len(params)
    arr = (Params * n)(*params)
    out = C.c_size_t()
    r = lib().cz_batch_workspace_size(n, arr, C.byref(out))
    if r != OK:
        raise CzError(r, "cz_batch_workspace_size")
    return out.value


def cz_compress_batch(b: BatchArgs, d_out_bytes: int, d_ws: int, ws_bytes: int, stream: int) -> int:
    return lib().cz_compress_batch(b.n, b.params, b.fields, b.outs, b.caps, d_out_bytes or None,
                                   d_ws, ws_bytes, stream or None)


def cz_batch_tune(b: BatchArgs, d_out_bytes: int, d_ws: int, ws_bytes: int, stream: int,
                  reps: int = 3) -> int:
    return lib().cz_batch_tune(b.n, b.params, b.fields, b.outs, b.caps, d_out_bytes or None,
                               d_ws, ws_bytes, stream or None, reps)


def cz_decompress(d_in: int, in_bytes: int, h_header, d_field: int, field_cap: int,
                  d_ws: int, ws_bytes: int, stream: int) -> int:
    hdr = None
    if h_header is not None:
        hdr = C.create_string_buffer(bytes(h_header[:HEADER_BYTES]), HEADER_BYTES)
    return lib().cz_decompress(d_in, in_bytes, hdr, d_field, field_cap, d_ws, ws_bytes,
                               stream or None)


def cz_read_header(h_in: bytes):
    buf = C.create_string_buffer(bytes(h_in[:HEADER_BYTES]), HEADER_BYTES)
    p = Params()
    t = C.c_double()
    r = lib().cz_read_header(buf, HEADER_BYTES, C.byref(p), C.byref(t))
    if r != OK:
        raise CzError(r, "cz_read_header")
    return p, t.value


def cz_status(d_ws: int, stream: int) -> int:
    return lib().cz_status(d_ws, stream or None)


def cz_strerror(code: int) -> str:
    return lib().cz_strerror(code).decode()


def cz_forward_dense(p: Params, d_field: int, d_coef: int, stream: int) -> int:
    return lib().cz_forward_dense(C.byref(p), d_field, d_coef, stream or None)


def cz_inverse_dense(p: Params, d_coef: int, d_field: int, stream: int) -> int:
    return lib().cz_inverse_dense(C.byref(p), d_coef, d_field, stream or None)


# ------------------------------------------------------------------ torch conveniences
def params_for(shape, dtype_is_f64: bool, block: int, kind, eps: float, eps_mode: int = EPS_REL,
               stage2: bool = True, range_: float = -1.0, bound_mode: int = BOUND_PAPER,
               fast: bool = False, zero_bits: int = 0, group: int = 1) -> Params:
    nz, ny, nx = shape
    if isinstance(kind, str):
        kind = KINDS[kind]
    flags = ((FLAG_FAST if fast else 0) | {0: 0, 4: FLAG_ZERO4, 8: FLAG_ZERO8}[int(zero_bits)]
             | GROUP_FLAGS[int(group)])
    return Params(nx, ny, nz, block, F64 if dtype_is_f64 else F32, kind, eps_mode,
                  int(stage2), int(bound_mode), flags, float(eps), float(range_))


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Workspace:
    """Device workspace sized for the largest parameter set seen so far."""

    def __init__(self, device=None):
        self.buf = None
        self.device = device

    def get(self, nbytes: int):
        import torch
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device or "cuda")
        return self.buf


def compress(field, block: int = 32, kind="w4", eps: float = 1e-3, eps_mode: int = EPS_REL,
             stage2: bool = True, range_: float = -1.0, out=None, ws: Workspace | None = None,
             stream=None, check: bool = True, bound_mode: int = BOUND_PAPER, fast: bool = False,
             zero_bits: int = 0, group: int = 1):
    """Compress a contiguous CUDA tensor [nz, ny, nx] (float32/float64).

    zero_bits = 4 / 8 zeroes that many least significant bits of every kept
    detail (bit zeroing Z4 / Z8).  group = 4 / 8 / 16 codes that many
    consecutive blocks as one aggregate chunk.  Returns (stream_tensor, nbytes_tensor); the
    stream is stream_tensor[:nbytes].  With check=True the call synchronises
    and raises on a device-side error.
    """
    import torch
    assert field.is_cuda and field.is_contiguous() and field.dim() == 3
    p = params_for(tuple(field.shape), field.dtype == torch.float64, block, kind, eps, eps_mode,
                   stage2, range_, bound_mode, fast, zero_bits, group)
    cap = cz_compress_bound(p)
    if out is None or out.numel() < cap:
        out = torch.empty(cap, dtype=torch.uint8, device=field.device)
    ws = ws or Workspace(field.device)
    wsb = ws.get(cz_workspace_size(p))
    nbytes = torch.zeros(1, dtype=torch.int64, device=field.device)
    s = _stream(stream)
    r = cz_compress(p, field.data_ptr(), out.data_ptr(), out.numel(), nbytes.data_ptr(),
                    wsb.data_ptr(), wsb.numel(), s)
    if r != OK:
        raise CzError(r, "cz_compress")
    if check:
        st = cz_status(wsb.data_ptr(), s)
        if st != OK:
            raise CzError(st, "cz_compress (device)")
    return out, nbytes


def decompress(stream_t, nbytes: int | None = None, header: bytes | None = None, out=None,
               ws: Workspace | None = None, stream=None, check: bool = True):
    """Decompress a CUDA uint8 stream tensor into a new (or given) field tensor."""
    import torch
    if header is None:
        header = stream_t[:HEADER_BYTES].cpu().numpy().tobytes()
    p, _ = cz_read_header(header)
    n = int(nbytes) if nbytes is not None else stream_t.numel()
    dt = torch.float64 if p.dtype == F64 else torch.float32
    if out is None:
        out = torch.empty((p.nz, p.ny, p.nx), dtype=dt, device=stream_t.device)
    ws = ws or Workspace(stream_t.device)
    wsb = ws.get(cz_workspace_size(p))
    s = _stream(stream)
    r = cz_decompress(stream_t.data_ptr(), n, header, out.data_ptr(),
                      out.numel() * out.element_size(), wsb.data_ptr(), wsb.numel(), s)
    if r != OK:
        raise CzError(r, "cz_decompress")
    if check:
        st = cz_status(wsb.data_ptr(), s)
        if st != OK:
            raise CzError(st, "cz_decompress (device)")
    return out


def decompress_blocks(stream_t, ids, nbytes: int | None = None, header: bytes | None = None, out=None,
                      ws: Workspace | None = None, stream=None, check: bool = True):
    """Random access: decode the blocks ids (a CUDA int32 tensor of block
    indices in x-fastest block order) into a new (or given) tensor of shape
    [len(ids), B, B, B]."""
    import torch
    if header is None:
        header = stream_t[:HEADER_BYTES].cpu().numpy().tobytes()
    p, _ = cz_read_header(header)
    assert ids.is_cuda and ids.dtype == torch.int32 and ids.is_contiguous()
    k = ids.numel()
    n = int(nbytes) if nbytes is not None else stream_t.numel()
    dt = torch.float64 if p.dtype == F64 else torch.float32
    B = p.block
    if out is None:
        out = torch.empty((k, B, B, B), dtype=dt, device=stream_t.device)
    ws = ws or Workspace(stream_t.device)
    need = C.c_size_t()
    r = lib().cz_decompress_blocks_workspace_size(C.byref(p), k, C.byref(need))
    if r != OK:
        raise CzError(r, "cz_decompress_blocks_workspace_size")
    wsb = ws.get(need.value)
    s = _stream(stream)
    hdr = C.create_string_buffer(bytes(header[:HEADER_BYTES]), HEADER_BYTES)
    r = lib().cz_decompress_blocks(stream_t.data_ptr(), n, hdr, ids.data_ptr() if k else None, k,
                                   out.data_ptr(), out.numel() * out.element_size(), wsb.data_ptr(), wsb.numel(),
                                   s or None)
    if r != OK:
        raise CzError(r, "cz_decompress_blocks")
    if check and k:
        st = cz_status(wsb.data_ptr(), s)
        if st != OK:
            raise CzError(st, "cz_decompress_blocks (device)")
    return out


def save_tuning(path: str):
    """Write the batch tuner's choices (cz_batch_knobs_export) to a JSON file."""
    n = C.c_size_t()
    r = lib().cz_batch_knobs_export(None, 0, C.byref(n))
    if r != OK:
        raise CzError(r, "cz_batch_knobs_export")
    buf = C.create_string_buffer(n.value)
    r = lib().cz_batch_knobs_export(C.cast(buf, C.c_void_p), n.value, C.byref(n))
    if r != OK:
        raise CzError(r, "cz_batch_knobs_export")
    with open(path, "w") as fh:
        fh.write(buf.value.decode())


def load_tuning(path: str):
    """Merge the batch tuner's choices from a JSON file (cz_batch_knobs_import)."""
    with open(path) as fh:
        r = lib().cz_batch_knobs_import(fh.read().encode())
    if r != OK:
        raise CzError(r, "cz_batch_knobs_import")


def compress_aos(cells, comps, block=None, kind="w3ai", eps=1e-3, eps_mode: int = EPS_REL, stage2: bool = True,
                 bound_mode: int = BOUND_PAPER, stream=None, check: bool = True):
    """Compress components comps of a contiguous CUDA cell array
    [nz, ny, nx, ncomp] (float32/float64) in one call (cz_compress_aos).
    block, kind and eps may be scalars or per-quantity lists.  Returns a
    list of (stream_tensor, nbytes) pairs, one per component."""
    import numpy as np
    import torch
    assert cells.is_cuda and cells.is_contiguous() and cells.dim() == 4
    nz, ny, nx, ncomp = cells.shape
    n = len(comps)
    f64 = cells.dtype == torch.float64
    per = lambda v: list(v) if isinstance(v, (list, tuple)) else [v] * n
    blocks = per(block) if block is not None else [16 if f64 else 32] * n
    params = [params_for((nz, ny, nx), f64, b, k, e, eps_mode, stage2, -1.0, bound_mode)
              for b, k, e in zip(blocks, per(kind), per(eps))]
    arr = (Params * n)(*params)
    caps = [cz_compress_bound(q) for q in params]
    outs = [torch.empty(c, dtype=torch.uint8, device=cells.device) for c in caps]
    nbytes = torch.zeros(n, dtype=torch.int64, device=cells.device)
    need = C.c_size_t()
    r = lib().cz_aos_workspace_size(n, arr, C.byref(need))
    if r != OK:
        raise CzError(r, "cz_aos_workspace_size")
    ws = torch.empty(need.value, dtype=torch.uint8, device=cells.device)
    comps_a = np.ascontiguousarray(np.asarray(comps, dtype=np.int32))
    s = _stream(stream)
    r = lib().cz_compress_aos(n, arr, cells.data_ptr(), ncomp, comps_a.ctypes.data_as(C.c_void_p),
                              (C.c_void_p * n)(*[o.data_ptr() for o in outs]), (C.c_size_t * n)(*caps),
                              nbytes.data_ptr(), ws.data_ptr(), ws.numel(), s or None)
    if r != OK:
        raise CzError(r, "cz_compress_aos")
    if check:
        st = cz_status(ws.data_ptr(), s)
        if st != OK:
            raise CzError(st, "cz_compress_aos (device)")
    return [(outs[i], nbytes[i]) for i in range(n)]


class Cache:
    """Decoded-block cache (cz_cache_*): fetch(stream_t, ids) returns the
    tiles of blocks ids (a host sequence of block indices) as a new (or
    given) CUDA tensor [len(ids), B, B, B], decoding only the blocks the
    cache does not hold."""

    def __init__(self, capacity: int, block: int, f64: bool = False):
        self.capacity, self.block, self.f64 = capacity, block, f64
        h = C.c_void_p()
        r = lib().cz_cache_create(capacity, block, F64 if f64 else F32, C.byref(h))
        if r != OK:
            raise CzError(r, "cz_cache_create")
        self._h = h
        self._ws = None

    def fetch(self, stream_t, ids, nbytes: int | None = None, header: bytes | None = None, out=None,
              ws: Workspace | None = None, stream=None, check: bool = True):
        import numpy as np
        import torch
        if header is None:
            header = stream_t[:HEADER_BYTES].cpu().numpy().tobytes()
        header = bytes(header[:HEADER_BYTES])
        ids = np.ascontiguousarray(np.asarray(ids, dtype=np.int32))
        k = int(ids.size)
        n = int(nbytes) if nbytes is not None else stream_t.numel()
        B = self.block
        dt = torch.float64 if self.f64 else torch.float32
        if out is None:
            out = torch.empty((k, B, B, B), dtype=dt, device=stream_t.device)
        ws = ws or self._ws or Workspace(stream_t.device)
        self._ws = ws
        # the parsed header, its C copy and the workspace size per request
        # size, kept for the stream last seen
        if getattr(self, "_hdr_key", None) != header:
            self._hdr_key = header
            self._hdr_p, _ = cz_read_header(header)
            self._hdr_c = C.create_string_buffer(header, HEADER_BYTES)
            self._need = {}
        if k not in self._need:
            need = C.c_size_t()
            r = lib().cz_decompress_blocks_workspace_size(C.byref(self._hdr_p), max(k, 1), C.byref(need))
            if r != OK:
                raise CzError(r, "cz_decompress_blocks_workspace_size")
            self._need[k] = need.value
        wsb = ws.get(self._need[k])
        s = _stream(stream)
        hdr = self._hdr_c
        hits = C.c_int(0)
        r = lib().cz_cache_fetch(self._h, stream_t.data_ptr(), n, hdr,
                                 ids.ctypes.data_as(C.c_void_p) if k else None, k, out.data_ptr(),
                                 out.numel() * out.element_size(), wsb.data_ptr(), wsb.numel(), s or None,
                                 C.byref(hits))
        if r != OK:
            raise CzError(r, "cz_cache_fetch")
        if check and k:
            st = cz_status(wsb.data_ptr(), s)
            if st != OK:
                raise CzError(st, "cz_cache_fetch (device)")
        return out, hits.value

    def clear(self):
        r = lib().cz_cache_clear(self._h)
        if r != OK:
            raise CzError(r, "cz_cache_clear")

    def stats(self):
        held, hits, misses = C.c_int(), C.c_longlong(), C.c_longlong()
        r = lib().cz_cache_stats(self._h, C.byref(held), C.byref(hits), C.byref(misses))
        if r != OK:
            raise CzError(r, "cz_cache_stats")
        return held.value, hits.value, misses.value

    def close(self):
        if getattr(self, "_h", None):
            lib().cz_cache_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def compress_batch(fields, block=None, kind="w3ai", eps=1e-3, eps_mode: int = EPS_REL,
                   stage2: bool = True, bound_mode: int = BOUND_PAPER, stream=None, check: bool = True,
                   tune: bool = False):
    """Compress a list of contiguous CUDA tensors in one batched call.

    block, kind and eps may be scalars or per-field lists (block defaults to
    32 for float32 and 16 for float64).  Returns a list of (stream_tensor,
    nbytes) pairs; stream i is out[i][:nbytes[i]].
    """
    import torch
    n = len(fields)
    per = lambda v: list(v) if isinstance(v, (list, tuple)) else [v] * n
    blocks = per(block) if block is not None else [16 if f.dtype == torch.float64 else 32 for f in fields]
    kinds, epss = per(kind), per(eps)
    params, caps, outs = [], [], []
    for f, b, k, e in zip(fields, blocks, kinds, epss):
        assert f.is_cuda and f.is_contiguous() and f.dim() == 3
        p = params_for(tuple(f.shape), f.dtype == torch.float64, b, k, e, eps_mode, stage2, -1.0,
                       bound_mode)
        params.append(p)
        cap = cz_compress_bound(p)
        caps.append(cap)
        outs.append(torch.empty(cap, dtype=torch.uint8, device=f.device))
    dev = fields[0].device
    nbytes = torch.zeros(n, dtype=torch.int64, device=dev)
    ws = torch.empty(cz_batch_workspace_size(params), dtype=torch.uint8, device=dev)
    b = BatchArgs(params, [f.data_ptr() for f in fields], [o.data_ptr() for o in outs], caps)
    s = _stream(stream)
    if tune:
        r = cz_batch_tune(b, nbytes.data_ptr(), ws.data_ptr(), ws.numel(), s)
        if r != OK:
            raise CzError(r, "cz_batch_tune")
    r = cz_compress_batch(b, nbytes.data_ptr(), ws.data_ptr(), ws.numel(), s)
    if r != OK:
        raise CzError(r, "cz_compress_batch")
    if check:
        st = cz_status(ws.data_ptr(), s)
        if st != OK:
            raise CzError(st, "cz_compress_batch (device)")
    return [(outs[i], nbytes[i]) for i in range(n)]


class Server:
    """The request server of the C ABI (cz_server_*): device pool of
    `budget_bytes`, `streams` CUDA streams, continuous admission."""

    def __init__(self, budget_bytes: int, streams: int = 4):
        self.h = C.c_void_p()
        r = lib().cz_server_create(int(budget_bytes), int(streams), C.byref(self.h))
        if r != OK:
            raise CzError(r, "cz_server_create")

    def submit_compress(self, p: Params, d_field: int, d_out: int, out_cap: int, d_out_bytes: int) -> int:
        q = Request()
        q.op = OP_COMPRESS
        q.params = p
        q.d_in = d_field
        q.d_out = d_out
        q.out_cap = out_cap
        q.d_out_bytes = d_out_bytes or None
        return self._submit(q)

    def submit_decompress(self, d_stream: int, nbytes: int, header: bytes, d_field: int, field_cap: int) -> int:
        q = Request()
        q.op = OP_DECOMPRESS
        q.d_in = d_stream
        q.in_bytes = nbytes
        C.memmove(q.h_header, bytes(header[:HEADER_BYTES]), HEADER_BYTES)
        q.d_out = d_field
        q.out_cap = field_cap
        return self._submit(q)

    def _submit(self, q) -> int:
        t = C.c_uint64()
        r = lib().cz_server_submit(self.h, C.byref(q), C.byref(t))
        if r != OK:
            raise CzError(r, "cz_server_submit")
        return t.value

    def poll(self, ticket: int):
        st, res, lat = C.c_int(), C.c_int(), C.c_double()
        r = lib().cz_server_poll(self.h, ticket, C.byref(st), C.byref(res), C.byref(lat))
        if r != OK:
            raise CzError(r, "cz_server_poll")
        return st.value, res.value, lat.value

    def wait(self, ticket: int):
        res, lat = C.c_int(), C.c_double()
        r = lib().cz_server_wait(self.h, ticket, C.byref(res), C.byref(lat))
        if r != OK:
            raise CzError(r, "cz_server_wait")
        return res.value, lat.value

    def close(self):
        if self.h:
            lib().cz_server_destroy(self.h)
            self.h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def stream_concat(streams) -> bytes:
    """Join slab streams (bytes, in z order) into the whole field's stream
    (cz_stream_concat); host-side, no GPU needed."""
    n = len(streams)
    bufs = [C.create_string_buffer(bytes(s), len(s)) for s in streams]
    ptrs = (C.c_void_p * n)(*[C.cast(b, C.c_void_p) for b in bufs])
    sizes = (C.c_size_t * n)(*[len(s) for s in streams])
    total = C.c_size_t()
    r = lib().cz_stream_concat(n, ptrs, sizes, None, 0, C.byref(total))
    if r != OK:
        raise CzError(r, "cz_stream_concat")
    out = C.create_string_buffer(total.value)
    r = lib().cz_stream_concat(n, ptrs, sizes, out, total.value, C.byref(total))
    if r != OK:
        raise CzError(r, "cz_stream_concat")
    return out.raw[:total.value]
