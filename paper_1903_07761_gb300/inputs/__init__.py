"""Seeded synthetic workload generators (host C, OpenMP over z-planes).

They stand in for the paper's cloud-cavitation snapshots (Sec. 3.1), which are
not available: a Gaussian-bubble field (128^3 small case) and the gas
fraction / density / pressure of a cloud of tanh-interface bubbles with
low-wavenumber pressure modes (512^3 multi-field and 1024^3 / 768^3 large
cases).  The recipes are documented in ``czgen.c``.  This module holds none of
the codec's arithmetic; the same bytes go to the GPU library and to the oracle.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libczgen.so")
_lock = threading.Lock()
_lib = None

GAUSS, ALPHA, RHO, P = 0, 1, 2, 3
RECIPES = {"gauss": GAUSS, "alpha": ALPHA, "rho": RHO, "p": P}


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    src = os.path.join(_HERE, "czgen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fopenmp",
                        "-fPIC", "-shared", "-o", tmp, src, "-lm"], check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            L.czgen_field.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                      C.c_uint64, C.c_int, C.c_void_p]
            L.czgen_field.restype = C.c_int
            _lib = L
    return _lib


def field(recipe, shape, dtype=np.float32, seed: int = 0, nbubbles: int = 200,
          out: np.ndarray | None = None) -> np.ndarray:
    """Generate a field of ``shape`` = (nz, ny, nx) in C order."""
    if isinstance(recipe, str):
        recipe = RECIPES[recipe]
    nz, ny, nx = shape
    dtype = np.dtype(dtype)
    if out is None:
        out = np.empty(shape, dtype)
    assert out.shape == tuple(shape) and out.dtype == dtype and out.flags.c_contiguous
    r = _load().czgen_field(recipe, 1 if dtype == np.float64 else 0, nx, ny, nz,
                            seed & (2 ** 64 - 1), nbubbles,
                            out.ctypes.data_as(C.c_void_p))
    if r != 0:
        raise RuntimeError("czgen_field failed")
    return out


def config0(seed: int = 0) -> np.ndarray:
    """128^3 FP32 Gaussian-bubble field (the small W4 case)."""
    return field(GAUSS, (128, 128, 128), np.float32, seed)


def cavitation(which: str, n: int, dtype=np.float32, seed: int = 1000,
               nbubbles: int = 200) -> np.ndarray:
    """alpha / rho / p of the bubble-cloud recipe on an n^3 domain."""
    return field(RECIPES[which], (n, n, n), dtype, seed, nbubbles)
