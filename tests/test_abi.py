"""The C ABI without a GPU: the library builds and loads, exports every
function that include/cz.h declares, and its host-side logic (parameter
checks, stream bound, header parsing, error texts) behaves as declared.
No call here launches a kernel.
"""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "cz.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const\s+char\s*\*)\s*(cz_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def cz():
    from paper_1903_07761_gb300 import cz as mod
    mod.lib()
    return mod


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("cz_compress", "cz_decompress", "cz_compress_bound", "cz_workspace_size",
              "cz_read_header", "cz_status", "cz_strerror", "cz_forward_dense",
              "cz_inverse_dense", "cz_compress_noalloc", "cz_noalloc_status"):
        assert n in names


def test_library_exports_every_declared_function(cz):
    from paper_1903_07761_gb300 import _build
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        assert hasattr(cz.lib(), n)


def test_strerror_covers_every_code(cz):
    texts = {code: cz.cz_strerror(code) for code in
             (cz.OK, cz.ERR_ARG, cz.ERR_CAPACITY, cz.ERR_CORRUPT, cz.ERR_TIMEOUT, cz.ERR_CUDA, cz.ERR_BUDGET)}
    assert all(texts.values())
    assert len(set(texts.values())) == len(texts)


@pytest.mark.parametrize("dims,block,f64", [((32, 32, 32), 32, False), ((16, 48, 32), 16, True),
                                            ((8, 8, 24), 8, False), ((32, 32, 64), 32, True),
                                            ((64, 64, 64), 64, False)])
def test_compress_bound_covers_the_worst_stream(cz, dims, block, f64):
    p = cz.params_for(dims, f64, block, "w4", 0.0, cz.EPS_REL, True, 1.0)
    bound = cz.cz_compress_bound(p)
    assert bound >= O.compress_bound(dims, block, np.float64 if f64 else np.float32)
    # white noise at eps = 0 keeps every coefficient: the stream must fit
    rng = np.random.default_rng(5)
    f = rng.standard_normal(dims).astype(np.float64 if f64 else np.float32)
    for st2 in (True, False):
        s = O.compress(f, block, O.W4, 0.0, O.EPS_REL, st2)
        assert len(s) <= bound


def test_invalid_parameters_are_refused_on_the_host(cz):
    bad = [((32, 32, 48), 32, False), ((16, 16, 16), 12, False), ((32, 32, 24), 32, True),
           ((0, 32, 32), 32, False), ((64, 64, 64), 64, True), ((64, 64, 64), 128, False)]
    for dims, block, f64 in bad:
        p = cz.params_for(dims, f64, block, "w4", 1e-3, cz.EPS_REL, True, 1.0)
        with pytest.raises(cz.CzError) as e:
            cz.cz_compress_bound(p)
        assert e.value.code == cz.ERR_ARG
    p = cz.params_for((32, 32, 32), False, 32, "w4", -1.0, cz.EPS_REL, True, 1.0)
    with pytest.raises(cz.CzError):
        cz.cz_compress_bound(p)
    p = cz.params_for((32, 32, 32), False, 32, "w4", float("nan"), cz.EPS_REL, True, 1.0)
    with pytest.raises(cz.CzError):
        cz.cz_compress_bound(p)
    # null buffers are refused before any CUDA call
    p = cz.params_for((32, 32, 32), False, 32, "w4", 1e-3, cz.EPS_REL, True, 1.0)
    assert cz.cz_compress(p, 0, 0, 1 << 20, 0, 0, 1 << 20, 0) == cz.ERR_ARG
    assert cz.lib().cz_compress_noalloc(C.byref(cz.params_for((32, 32, 48), False, 32, "w4", 1e-3)),
                                        None, None, 0, None, None) == cz.ERR_ARG
    # a valid shape with null or misaligned buffers: refused before the
    # no-alloc entry point looks up its workspace (a CUDA call)
    ok = C.byref(cz.params_for((128, 128, 128), False, 32, "w4", 1e-3))
    assert cz.lib().cz_compress_noalloc(ok, None, None, 1 << 20, None, None) == cz.ERR_ARG
    assert cz.lib().cz_compress_noalloc(ok, 0x1000, None, 1 << 20, None, None) == cz.ERR_ARG
    assert cz.lib().cz_compress_noalloc(ok, 0x1008, 0x2000, 1 << 20, None, None) == cz.ERR_ARG


def test_read_header_of_an_oracle_stream(cz):
    rng = np.random.default_rng(3)
    f = rng.standard_normal((16, 32, 48)).astype(np.float32)
    s = O.compress(f, 16, O.W3AI, 1e-2, O.EPS_REL, True)
    p, t = cz.cz_read_header(s[:cz.HEADER_BYTES])
    assert (p.nx, p.ny, p.nz, p.block, p.dtype, p.kind, p.stage2) == (48, 32, 16, 16, cz.F32, cz.W3AI, 1)
    assert p.eps == 1e-2 and p.eps_mode == cz.EPS_REL
    h = O.read_header(s)
    assert t == h["t"]
    assert p.range == h["range"]
    bad = bytearray(s[:cz.HEADER_BYTES])
    bad[0] ^= 1  # magic
    with pytest.raises(cz.CzError) as e:
        cz.cz_read_header(bytes(bad))
    assert e.value.code == cz.ERR_CORRUPT
    bad = bytearray(s[:cz.HEADER_BYTES])
    bad[28] ^= 1  # block count disagrees with the dims
    with pytest.raises(cz.CzError):
        cz.cz_read_header(bytes(bad))


def test_group_flags_are_checked(cz):
    """Aggregate chunks: stage 2 only, and G times the largest block
    payload at most CZ_GROUP_MAX_BYTES (1792 KiB)."""
    def bound(shape, f64, block, group, stage2=True):
        p = cz.params_for(shape, f64, block, "w3ai", 1e-3, cz.EPS_REL, stage2, 1.0, group=group)
        return cz.cz_compress_bound(p)

    s = (64, 64, 64)
    for block, f64, ok in ((32, False, (4, 8)), (32, True, (4,)), (16, False, (4, 8, 16)),
                           (16, True, (4, 8, 16)), (8, True, (4, 8, 16)), (64, False, ())):
        for g in (4, 8, 16):
            if g in ok:
                assert bound(s, f64, block, g) > 0
            else:
                with pytest.raises(cz.CzError) as e:
                    bound(s, f64, block, g)
                assert e.value.code == cz.ERR_ARG
    with pytest.raises(cz.CzError) as e:
        bound(s, False, 16, 4, stage2=False)
    assert e.value.code == cz.ERR_ARG


def test_batched_calls_refuse_group_flags_on_the_host(cz):
    """Batched launches take no aggregate chunks: refused before any CUDA
    call (the device pointers below are never touched)."""
    p = cz.params_for((32, 32, 64), False, 16, "w3ai", 1e-3, group=4)
    with pytest.raises(cz.CzError) as e:
        cz.cz_batch_workspace_size([p])
    assert e.value.code == cz.ERR_ARG
    b = cz.BatchArgs([p], [1 << 20], [2 << 20], [1 << 20])
    assert cz.cz_compress_batch(b, 0, 3 << 20, 1 << 20, 0) == cz.ERR_ARG


def test_read_header_of_an_oracle_group_stream(cz):
    f = np.random.default_rng(5).standard_normal((32, 32, 48)).astype(np.float32)
    for g, flag in ((4, cz.FLAG_GROUP4), (8, cz.FLAG_GROUP8), (16, cz.FLAG_GROUP16)):
        s = O.compress(f, 8, O.W4, 1e-2, group=g, zbits=4)
        p, _ = cz.cz_read_header(s[:cz.HEADER_BYTES])
        assert p.flags == flag | cz.FLAG_ZERO4


def test_strict_divisor_equals_the_oracles(cz):
    """The library computes the strict-bound divisor C on the host in the
    same operation order as the oracle; equal C gives equal thresholds."""
    L = cz.lib()
    L.czi_synthesis_norm.argtypes = [C.c_int, C.c_int]
    L.czi_synthesis_norm.restype = C.c_double
    for kind in (O.W4, O.W4LI, O.W3AI):
        for B in (8, 16, 32, 64):
            assert L.czi_synthesis_norm(kind, B) == O.synthesis_norm(kind, B)


def test_bound_mode_and_flags_are_checked(cz):
    p = cz.params_for((32, 32, 32), False, 32, "w4", 1e-3, cz.EPS_REL, True, 1.0, bound_mode=2)
    with pytest.raises(cz.CzError):
        cz.cz_compress_bound(p)
    p = cz.params_for((32, 32, 32), False, 32, "w4", 1e-3, cz.EPS_REL, True, 1.0)
    p.flags = 32  # unknown flag
    with pytest.raises(cz.CzError):
        cz.cz_compress_bound(p)
    p.flags = cz.FLAG_ZERO4 | cz.FLAG_ZERO8  # one zeroing width at most
    with pytest.raises(cz.CzError):
        cz.cz_compress_bound(p)
    for f in (cz.FLAG_ZERO4, cz.FLAG_ZERO8):
        p.flags = f
        assert cz.cz_compress_bound(p) > 0
    # the fast build: W3ai only (W4 / W4li miss its 0.01 dB PSNR gate)
    for kind in ("w4", "w4li", "w3ai"):
        for f in (cz.FLAG_FAST, cz.FLAG_FAST | cz.FLAG_ZERO8):
            p = cz.params_for((32, 32, 32), False, 32, kind, 1e-3, cz.EPS_REL, True, 1.0)
            p.flags = f
            if kind == "w3ai":
                assert cz.cz_compress_bound(p) > 0
            else:
                with pytest.raises(cz.CzError) as e:
                    cz.cz_compress_bound(p)
                assert e.value.code == cz.ERR_ARG
    p = cz.params_for((32, 32, 32), False, 32, "w4", 1e-3, cz.EPS_REL, True, 1.0,
                      bound_mode=cz.BOUND_STRICT, zero_bits=8)  # the strict bound excludes zeroing
    with pytest.raises(cz.CzError):
        cz.cz_compress_bound(p)


def test_struct_layouts_match_the_header(cz, tmp_path):
    """ctypes mirrors of cz_params / cz_request have the C layout."""
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "cz.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(cz_params), sizeof(cz_request),'
                   ' offsetof(cz_params, eps), offsetof(cz_request, h_header), offsetof(cz_request, d_out));'
                   'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [C.sizeof(cz.Params), C.sizeof(cz.Request), cz.Params.eps.offset, cz.Request.h_header.offset,
            cz.Request.d_out.offset]
    assert got == want


def test_cache_arguments_are_refused_before_any_cuda_call(cz):
    """cz_cache_create / cz_cache_fetch check their arguments on the host
    before touching the device (so this runs without a GPU)."""
    h = C.c_void_p()
    for cap, B, dt in ((0, 32, cz.F32), (4, 12, cz.F32), (4, 32, 7)):
        assert cz.lib().cz_cache_create(cap, B, dt, C.byref(h)) == cz.ERR_ARG
        assert not h.value
    hits = C.c_int(5)
    assert cz.lib().cz_cache_fetch(None, None, 0, None, None, 0, None, 0, None, 0, None, C.byref(hits)) == cz.ERR_ARG
    assert hits.value == 0
    assert cz.lib().cz_cache_clear(None) == cz.ERR_ARG
    assert cz.lib().cz_cache_stats(None, None, None, None) == cz.ERR_ARG


def test_aos_arguments_are_refused_before_any_cuda_call(cz):
    """cz_aos_workspace_size / cz_compress_aos refuse an empty call and
    quantities of different field shapes on the host."""
    need = C.c_size_t()
    assert cz.lib().cz_aos_workspace_size(0, None, C.byref(need)) == cz.ERR_ARG
    a = cz.params_for((32, 32, 32), False, 32, "w4", 1e-3)
    b = cz.params_for((32, 32, 64), False, 32, "w4", 1e-3)
    arr = (cz.Params * 2)(a, b)
    assert cz.lib().cz_aos_workspace_size(2, arr, C.byref(need)) == cz.ERR_ARG
    comps = (C.c_int32 * 2)(0, 1)
    assert cz.lib().cz_compress_aos(2, arr, None, 4, comps, None, None, None, None, 0, None) == cz.ERR_ARG


def test_batch_tuner_choices_round_trip_through_json(cz, tmp_path):
    """cz_batch_knobs_export / _import (host only): choices written by one
    process are read back by another; an entry replaces the one with its
    signature; version 1 texts (before the scan-granularity and kernel-family
    knobs) still load, with tiles of 128 chunks and the register-resident
    kernels; malformed texts are refused and change nothing."""
    import json
    text = json.dumps({"format": "cz-batch-knobs", "version": 2, "entries": [
        {"signature": "00000000000000ab", "s1_balanced": 1, "s2_div": 2, "place_tile": 64, "slab": 1},
        {"signature": "fedcba9876543210", "s1_balanced": 0, "s2_div": 1, "place_tile": 256, "slab": 0}]}, indent=2)
    src = tmp_path / "in.json"
    src.write_text(text)
    cz.load_tuning(str(src))
    dst = tmp_path / "out.json"
    cz.save_tuning(str(dst))
    d = json.loads(dst.read_text())
    assert d["format"] == "cz-batch-knobs" and d["version"] == 2

    def entries():
        return {e["signature"]: (e["s1_balanced"], e["s2_div"], e["place_tile"], e["slab"])
                for e in json.loads(dst.read_text())["entries"]}
    got = entries()
    assert got["00000000000000ab"] == (1, 2, 64, 1) and got["fedcba9876543210"] == (0, 1, 256, 0)
    L = cz.lib()
    assert L.cz_batch_knobs_import(b'{"format":"cz-batch-knobs","version":1,"entries":'
                                   b'[{"signature":"ab","s1_balanced":0,"s2_div":4}]}') == cz.OK
    cz.save_tuning(str(dst))
    got = entries()
    assert got["00000000000000ab"] == (0, 4, 128, 0) and got["fedcba9876543210"] == (0, 1, 256, 0)
    before = dst.read_text()
    for bad in (b"{}", b'{"format": "other", "version": 1, "entries": []}',
                b'{"format": "cz-batch-knobs", "version": 3, "entries": []}',
                b'{"format": "cz-batch-knobs", "version": 1, "entries": [{"signature": "xyz", "s1_balanced": 0, "s2_div": 1}]}',
                b'{"format": "cz-batch-knobs", "version": 1, "entries": [{"signature": "ab", "s1_balanced": 0, "s2_div": 0}]}',
                b'{"format": "cz-batch-knobs", "version": 1, "entries": [{"signature": "ab", "s1_balanced": 2, "s2_div": 1}]}',
                b'{"format": "cz-batch-knobs", "version": 2, "entries": [{"signature": "ab", "s1_balanced": 0, "s2_div": 1}]}',
                b'{"format": "cz-batch-knobs", "version": 2, "entries": [{"signature": "ab", "s1_balanced": 0, "s2_div": 1, '
                b'"place_tile": 100, "slab": 0}]}',
                b'{"format": "cz-batch-knobs", "version": 2, "entries": [{"signature": "ab", "s1_balanced": 0, "s2_div": 1, '
                b'"place_tile": 64, "slab": 2}]}',
                b'{"format": "cz-batch-knobs", "version": 1, "entries": [{"signature": "cd", "s1_balanced": 0, "s2_div": 1}'):
        assert L.cz_batch_knobs_import(bad) == cz.ERR_ARG, bad
    cz.save_tuning(str(dst))
    assert dst.read_text() == before


def test_read_header_refuses_or_parses_every_mutated_header(cz):
    """Thousands of headers with one to three bytes changed: the parser
    either refuses with CZ_ERR_CORRUPT or returns parameters that pass the
    parameter checks (block edge, dims a multiple of it, codes in range, the
    block count equal to the dims').  A change confined to bytes it does not
    read (the level count, min/max, sizes, padding) leaves the parameters
    as they were."""
    f = np.random.default_rng(5).standard_normal((32, 64, 96)).astype(np.float32)
    s = O.compress(f, 32, O.W4LI, 1e-3, O.EPS_REL, True)[:cz.HEADER_BYTES]
    p0, t0 = cz.cz_read_header(s)
    fields = lambda p: (p.nx, p.ny, p.nz, p.block, p.dtype, p.kind, p.stage2, p.eps_mode, p.bound_mode,
                        p.flags, p.eps, p.range)
    ignored = {25} | set(range(40, 64)) | set(range(72, 128))
    rng = np.random.default_rng(11)
    accepted = refused = 0
    for _ in range(3000):
        h = bytearray(s)
        pos = rng.choice(cz.HEADER_BYTES, size=int(rng.integers(1, 4)), replace=False)
        for q in pos:
            h[q] ^= int(rng.integers(1, 256))
        try:
            p, _ = cz.cz_read_header(bytes(h))
        except cz.CzError as e:
            assert e.code == cz.ERR_CORRUPT, (pos, e.code)
            assert not set(pos.tolist()) <= ignored, pos
            refused += 1
            continue
        accepted += 1
        if set(pos.tolist()) <= ignored:
            assert fields(p) == fields(p0), pos
            continue
        assert p.block in (8, 16, 32, 64) and (p.block != 64 or p.dtype == cz.F32)
        assert all(n > 0 and n % p.block == 0 for n in (p.nx, p.ny, p.nz))
        assert p.dtype in (cz.F32, cz.F64) and p.kind in (cz.W4, cz.W4LI, cz.W3AI)
        assert p.stage2 in (0, 1) and p.eps_mode in (cz.EPS_REL, cz.EPS_ABS)
        assert p.bound_mode in (cz.BOUND_PAPER, cz.BOUND_STRICT) and p.eps >= 0
        nb = int.from_bytes(bytes(h[28:32]), "little")
        assert nb == (p.nx // p.block) * (p.ny // p.block) * (p.nz // p.block)
    assert accepted > 0 and refused > 0
    # shorter than a header: refused as an argument error
    buf = C.create_string_buffer(s, cz.HEADER_BYTES)
    assert cz.lib().cz_read_header(buf, cz.HEADER_BYTES - 1, C.byref(cz.Params()), None) == cz.ERR_ARG
