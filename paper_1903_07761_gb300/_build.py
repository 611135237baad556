"""Build the CUDA library libcz.so in-tree for sm_103a (GB300).

The kernels are instantiated once per (element type, block edge) in separate
translation units compiled in parallel, then linked with the host-side C ABI
into ``paper_1903_07761_gb300/_lib/libcz.so`` (CUDA runtime linked
statically).  Rebuilds only when a source is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_lib")
BUILD_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libcz.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-fast-math",
           "-Xcompiler", "-ffp-contract=off",
           "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]

# (type, block) instantiations of the kernels
INST = [("float", "f32", 8), ("float", "f32", 16), ("float", "f32", 32), ("float", "f32", 64),
        ("double", "f64", 8), ("double", "f64", 16), ("double", "f64", 32)]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcz.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*")) +
                  [os.path.join(ROOT, "include", "cz.h")])


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def _jobs(verbose_ptxas: bool):
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    jobs = []
    for fast in (False, True):
        for ctype, tname, b in INST:
            obj = os.path.join(BUILD_DIR, f"cz_inst_{tname}_b{b}{'_fast' if fast else ''}.o")
            cmd = [nvcc(), *ARCH, *NVFLAGS, *extra, f"-DCZ_T={ctype}", f"-DCZ_TNAME={tname}",
                   f"-DCZ_B={b}", *(["-DCZ_FAST"] if fast else []), "-c", os.path.join(CSRC, "cz_inst.cu"),
                   "-o", obj]
            jobs.append((obj, cmd))
    for name in ("cz_api", "cz_noalloc", "cz_serve", "cz_cache"):
        obj = os.path.join(BUILD_DIR, f"{name}.o")
        jobs.append((obj, [nvcc(), *ARCH, *NVFLAGS, *extra, "-c", os.path.join(CSRC, f"{name}.cu"),
                           "-o", obj]))
    return jobs


def build(force: bool = False, verbose_ptxas: bool = False, quiet: bool = True) -> str:
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    os.makedirs(OUT_DIR, exist_ok=True)
    jobs = _jobs(verbose_ptxas)

    def run(job):
        obj, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        return obj, cmd, r

    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(run, jobs))
    for obj, cmd, r in results:
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}")
        if verbose_ptxas or not quiet:
            sys.stderr.write(r.stderr)
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc(), *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp,
            *[obj for obj, _, _ in results]]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("link of libcz.so failed")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, quiet=False)
    print(LIB)
