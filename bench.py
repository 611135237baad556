#!/usr/bin/env python3
"""Benchmark of the GB300 wavelet codec (one JSON line on stdout, rank 0).

Workload: the bandwidth-bound large case -- a 1024^3 FP32 pressure field of
the synthetic bubble-cloud recipe (200 tanh-interface bubbles, eight
low-wavenumber pressure modes, a pressure drop inside the bubbles), cut into
32^3 blocks, eps = 1e-3 of the field range, stage 2 on.  It stands in for
the paper's cloud-cavitation pressure snapshots (Sec. 3.1, Sec. 4.3 uses
1024^3 per node).  One step is the whole hot path on that field:
  a0 min/max -> compress (transform, threshold, mask, compaction, stage 2,
  look-back offsets) -> decompress (stage-2 inverse, scatter, inverse
  transform),
all through the C ABI (cz_compress / cz_decompress).  The field (4 GiB) is
larger than L2, so no L2 flush is needed between steps.

value = field bytes / (compress + decompress time) in GB/s, whole job over
N ranks (each rank compresses its own field; no data-path collective).

--impl reference times the CPU oracle (the plain C reference written from
the paper) on host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compress+decompress GB/s & %HBM peak @eps=1e-3 1024^3 FP32; served p50/p99 ms"
UNIT = "GB/s"


# ------------------------------------------------------------------ helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the sources of the register-resident kernels and their launches (the
# kernels the traffic keys describe)
KERNEL_SOURCES = ("cz_compress.cuh", "cz_device.cuh", "cz_inst.cu", "cz_pair.cuh")


def csrc_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1903_07761_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(d, name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_launch(kernel: str, units: float):
    """DRAM bytes of one launch from the committed ncu summary, if the
    kernel sources are unchanged since it was taken (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        e = d[kernel]
        if e.get("csrc_sha") != csrc_hash():
            return None
        return e["dram_bytes_per_unit"] * units
    except Exception:
        return None


def rank_max(values, device):
    """Element-wise maximum of a list of floats over all ranks (the job's
    time is the slowest rank's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def replica_throughput(world, bytes_per_rank, ms_per_step):
    """Whole-job GB/s: every rank processes its own field in each step."""
    return world * bytes_per_rank / (ms_per_step * 1e-3) / 1e9


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.path = None
        self.dev = device_index

    def start(self):
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.dev).uuid)
            ident = uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"
            fd, self.path = tempfile.mkstemp(prefix="czclk", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", ident, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            with open(self.path) as fh:
                for line in fh:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 8:
                        rows.append(parts)
            os.unlink(self.path)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        smax = [num(r[1]) for r in rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ workload
def workload_config(n: int, B: int, kind: str, world: int) -> dict:
    """The `config` object of the JSON line (the same for both arms)."""
    return {"workload": f"p-field {n}^3 FP32, {B}^3 blocks, {kind}, eps=1e-3*range, stage2 on, "
                        f"range computed by the codec",
            "global_batch": world, "field_bytes": 4 * n ** 3,
            "l2": f"inputs larger than L2 ({4 * n ** 3 / 2**30:.0f} GiB field per step), no flush needed",
            "parallelism": f"replicas x{world} (independent fields, no collective)"}


def make_field(n: int, seed: int):
    from paper_1903_07761_gb300 import inputs
    return inputs.cavitation("p", n, seed=seed)


def cpu_oracle_run(field_np, block, kind, eps, slabs, rng):
    """Oracle compress + decompress of the first `slabs` block-rows of z
    (threshold from the full field's range).  Returns (bytes, seconds)."""
    import oracle as O
    sample = field_np[: slabs * block]
    t0 = time.perf_counter()
    s = O.compress(sample, block, kind, eps, range_=rng)
    O.decompress(s)
    return sample.nbytes, time.perf_counter() - t0


# the same oracle on all host cores: independent tasks (a z-slab of blocks,
# a quarter of its rows of blocks each) in worker processes started with
# `spawn` (the parent holds a CUDA context), the sample shared through a
# memory map
_ORACLE_SHARED = None


def _oracle_worker_init(path, shape, dtype_str):
    global _ORACLE_SHARED
    import numpy as np
    import oracle  # noqa: F401  (load the oracle before the clock starts)
    _ORACLE_SHARED = np.memmap(path, dtype=np.dtype(dtype_str), mode="r", shape=shape)


def _oracle_worker_ready(_):
    return os.getpid()


def _oracle_worker_task(a):
    import numpy as np
    import oracle as O
    fidx, z0, z1, y0, y1, block, kind, eps, rng = a
    sub = np.ascontiguousarray(_ORACLE_SHARED[fidx, z0:z1, y0:y1])
    s = O.compress(sub, block, kind, eps, range_=rng)
    O.decompress(s)
    return sub.nbytes


def _slab_tasks(shape, block, kind, eps, rng, fidx=0):
    """Independent oracle tasks over a field: z-slabs of one block row, each
    cut into (about) four y-ranges of whole blocks."""
    ny = shape[1]
    q = max(block, (ny // 4) // block * block)
    return [(fidx, z, z + block, y, min(y + q, ny), block, kind, eps, rng)
            for z in range(0, shape[0], block) for y in range(0, ny, q)]


def cpu_oracle_pool(fields, tasks):
    """Run oracle compress + decompress tasks (see _slab_tasks) over the
    given fields (equal shapes and type) on every host core.  Returns
    (bytes, seconds, cores)."""
    import multiprocessing as mp
    import shutil
    import numpy as np
    shape, dt = fields[0].shape, fields[0].dtype
    total = sum(f.nbytes for f in fields)
    d = "/dev/shm" if os.path.isdir("/dev/shm") and shutil.disk_usage("/dev/shm").free > 2 * total \
        else tempfile.gettempdir()
    fd, path = tempfile.mkstemp(dir=d, suffix=".oracle_sample")
    os.close(fd)
    try:
        mm = np.memmap(path, dtype=dt, mode="w+", shape=(len(fields),) + tuple(shape))
        for i, f in enumerate(fields):
            mm[i] = f
        mm.flush()
        del mm
        cores = os.cpu_count() or 1
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores, initializer=_oracle_worker_init,
                      initargs=(path, (len(fields),) + tuple(shape), dt.str)) as pool:
            pool.map(_oracle_worker_ready, range(cores))
            t0 = time.perf_counter()
            done = sum(pool.map(_oracle_worker_task, tasks, chunksize=1))
            secs = time.perf_counter() - t0
        return done, secs, cores
    finally:
        os.unlink(path)


def cpu_oracle_all_cores(field_np, block, kind, eps, slabs, rng):
    """Oracle compress + decompress of the first `slabs` block-rows of z on
    every host core.  Returns (bytes, seconds, cores)."""
    sample = field_np[: slabs * block]
    return cpu_oracle_pool([sample], _slab_tasks(sample.shape, block, kind, eps, rng))


def oracle_sweep_timing(n1: int = 512, seed1: int = 1000, slabs: int = 1, slabs_all: int = 2):
    """The oracle as it stands on the small Gaussian-bubble field (128^3, W4,
    eps 1e-3) and on the 512^3 bubble-cloud sweep, single-threaded and on all
    host cores.  The cloud runs take bounded samples: the first `slabs`
    z-slabs of blocks of the pressure field per kind at eps 1e-3 (one
    thread), and the first `slabs_all` z-slabs of every field for all 36
    runs of the sweep (all cores), each with the threshold of its full
    field.  (The oracle forms the W4li update weights from their exact
    fractions at every use, so W4li runs far slower than the other kinds.)"""
    import oracle as O
    from paper_1903_07761_gb300 import inputs
    out = {"cores_all": os.cpu_count() or 1}
    f0 = inputs.config0(seed=0)
    r0 = float(f0.max()) - float(f0.min())
    t0 = time.perf_counter()
    O.decompress(O.compress(f0, 32, O.W4, 1e-3, range_=r0))
    secs = time.perf_counter() - t0
    out["small_single"] = {"gbs": f0.nbytes / secs / 1e9, "seconds": secs, "cores": 1,
                           "what": "128^3 FP32 Gaussian bubbles, 32^3 blocks, W4, eps 1e-3, compress + decompress"}
    tasks0 = [(0, z, z + 32, y, y + 32, 32, O.W4, 1e-3, r0) for z in range(0, 128, 32) for y in range(0, 128, 32)]
    b, secs, cores = cpu_oracle_pool([f0], tasks0)
    out["small_all"] = {"gbs": b / secs / 1e9, "seconds": secs, "cores": cores}
    names = ("alpha", "rho", "p")
    fields = [inputs.cavitation(w, n1, seed=seed1) for w in names]
    rngs = [float(f.max()) - float(f.min()) for f in fields]
    single = {}
    smp = fields[2][: slabs * 32]
    for kname, kk in (("w4", O.W4), ("w4li", O.W4LI), ("w3ai", O.W3AI)):
        t0 = time.perf_counter()
        O.decompress(O.compress(smp, 32, kk, 1e-3, range_=rngs[2]))
        secs = time.perf_counter() - t0
        single[kname] = {"gbs": smp.nbytes / secs / 1e9, "seconds": secs}
    out["cloud_single_p_eps1e-3"] = {
        "per_kind": single, "cores": 1,
        "what": f"the first {slabs} z-slab(s) of 32^3 blocks ({smp.nbytes / 2**20:.0f} MiB) of the {n1}^3 "
                f"FP32 p-field, compress + decompress, one thread"}
    samples = [f[: slabs_all * 32] for f in fields]
    tasks = []
    for fi in range(3):
        for kk in (O.W4, O.W4LI, O.W3AI):
            for eps in (1e-2, 1e-3, 1e-4, 1e-5):
                tasks += _slab_tasks(samples[fi].shape, 32, kk, eps, rngs[fi], fidx=fi)
    b, secs, cores = cpu_oracle_pool(samples, tasks)
    out["cloud_all"] = {"gbs": b / secs / 1e9, "seconds": secs, "cores": cores,
                        "what": f"all 36 runs of the {n1}^3 sweep (3 fields x 3 kinds x 4 eps) on the first "
                                f"{slabs_all} z-slab(s) of each field ({samples[0].nbytes / 2**20:.0f} MiB), "
                                f"compress + decompress, {len(tasks)} tasks"}
    return out


# ------------------------------------------------------------------ GPU arm
def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1903_07761_gb300 import cz

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    kind = cz.KINDS[args.kind]
    n, B = args.n, args.block
    field_np = make_field(n, seed=2000 + rank)
    field = torch.from_numpy(field_np).to(dev)
    nbytes_field = field.numel() * field.element_size()
    p = cz.params_for(tuple(field.shape), False, B, kind, args.eps, cz.EPS_REL, True, -1.0)
    cap = cz.cz_compress_bound(p)
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    ws = torch.empty(cz.cz_workspace_size(p), dtype=torch.uint8, device=dev)
    nb = torch.zeros(1, dtype=torch.int64, device=dev)
    rec = torch.empty_like(field)
    stream = torch.cuda.current_stream(dev)
    s = stream.cuda_stream

    def compress_call(pp=p):
        r = cz.cz_compress(pp, field.data_ptr(), out.data_ptr(), cap, nb.data_ptr(),
                           ws.data_ptr(), ws.numel(), s)
        if r != cz.OK:
            raise cz.CzError(r, "cz_compress")

    compress_call()
    st = cz.cz_status(ws.data_ptr(), s)
    if st != cz.OK:
        raise cz.CzError(st, "cz_compress (device)")
    stream_len = int(nb.item())
    header = out[:cz.HEADER_BYTES].cpu().numpy().tobytes()
    hdr_c = cz.C.create_string_buffer(header, cz.HEADER_BYTES)

    def decompress_call():
        r = cz.lib().cz_decompress(out.data_ptr(), stream_len, hdr_c, rec.data_ptr(),
                                   nbytes_field, ws.data_ptr(), ws.numel(), s)
        if r != cz.OK:
            raise cz.CzError(r, "cz_decompress")

    lib = cz.lib()
    lib.czi_compress_marked.argtypes = [cz.C.POINTER(cz.Params), cz.C.c_void_p, cz.C.c_void_p,
                                        cz.C.c_size_t, cz.C.c_void_p, cz.C.c_void_p, cz.C.c_size_t,
                                        cz.C.c_void_p, cz.C.POINTER(cz.C.c_void_p)]
    lib.czi_compress_marked.restype = cz.C.c_int

    def compress_marked(marks):
        # cz_compress with events recorded between its kernels: marks[0]
        # before the stage kernel, [1] after it, [2] after stage 2, [3] after
        # the chunk copy (same launches as cz_compress)
        arr = (cz.C.c_void_p * 4)(*[m.cuda_event for m in marks[:4]])
        r = lib.czi_compress_marked(cz.C.byref(p), field.data_ptr(), out.data_ptr(), cap,
                                    nb.data_ptr(), ws.data_ptr(), ws.numel(), s, arr)
        if r != cz.OK:
            raise cz.CzError(r, "cz_compress")

    lib.czi_decompress_marked.argtypes = [cz.C.c_void_p, cz.C.c_size_t, cz.C.c_void_p, cz.C.c_void_p,
                                          cz.C.c_size_t, cz.C.c_void_p, cz.C.c_size_t, cz.C.c_void_p,
                                          cz.C.POINTER(cz.C.c_void_p)]
    lib.czi_decompress_marked.restype = cz.C.c_int

    def decompress_marked(mark):
        # cz_decompress with one event recorded right before the decode
        # kernel (after the stage-2 inverse launches; same launches)
        arr = (cz.C.c_void_p * 1)(mark.cuda_event)
        r = lib.czi_decompress_marked(out.data_ptr(), stream_len, hdr_c, rec.data_ptr(), nbytes_field,
                                      ws.data_ptr(), ws.numel(), s, arr)
        if r != cz.OK:
            raise cz.CzError(r, "cz_decompress")

    def step():
        compress_call()
        decompress_call()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    mk = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    for m in mk:
        for e in m:
            e.record(stream)  # create the events before the timed region
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for (e0, e1, e2), m in zip(ev, mk):
        e0.record(stream)
        compress_marked(m)
        e1.record(stream)
        decompress_marked(m[4])
        e2.record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    comp_ms = sum(a.elapsed_time(b) for a, b, _ in ev) / args.steps
    dec_ms = sum(b.elapsed_time(c) for _, b, c in ev) / args.steps
    # per-kernel durations inside the timed steps (same stream as the launches)
    range_ms = sum(e0.elapsed_time(m[0]) for (e0, _, _), m in zip(ev, mk)) / args.steps
    stage1_ms = sum(m[0].elapsed_time(m[1]) for m in mk) / args.steps
    stage2_ms = sum(m[1].elapsed_time(m[2]) for m in mk) / args.steps
    place_ms = sum(m[2].elapsed_time(m[3]) for m in mk) / args.steps
    unstage_ms = sum(e1.elapsed_time(m[4]) for (_, e1, _), m in zip(ev, mk)) / args.steps
    dec2_ms = sum(m[4].elapsed_time(e2) for (_, _, e2), m in zip(ev, mk)) / args.steps
    st = cz.cz_status(ws.data_ptr(), s)
    if st != cz.OK:
        raise cz.CzError(st, "device status after timed steps")
    stream_len = int(nb.item())

    # quality of the last step (measurement only)
    diff = (rec.double() - field.double())
    mse = float((diff * diff).mean().item())
    linf = float(diff.abs().max().item())
    fmin, fmax = float(field.min().item()), float(field.max().item())
    psnr = 20 * math.log10((fmax - fmin) / (2 * math.sqrt(mse))) if mse > 0 else float("inf")
    del diff

    # compression with the range supplied by the caller (no min/max pass):
    # algorithmic bytes N*s read + S written
    p_rng = cz.params_for(tuple(field.shape), False, B, kind, args.eps, cz.EPS_REL, True, fmax - fmin)
    rng_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
    compress_call(p_rng)
    for a_, b_ in rng_ev:
        a_.record(stream)
        compress_call(p_rng)
        b_.record(stream)
    torch.cuda.synchronize()
    st = cz.cz_status(ws.data_ptr(), s)
    if st != cz.OK:
        raise cz.CzError(st, "cz_compress with the range supplied (device)")
    rng_len = int(nb.item())
    rng_ms = statistics.median(a_.elapsed_time(b_) for a_, b_ in rng_ev)
    compress_range_supplied = {"ms": rng_ms, "gbs": nbytes_field / rng_ms / 1e6,
                               "hbm_frac": (nbytes_field + rng_len) / (rng_ms * 1e-3) / 1e9 / measured_peaks()[0],
                               "algorithmic_bytes": nbytes_field + rng_len, "stream_bytes": rng_len,
                               "what": "cz_compress with p.range = max - min given (no min/max pass), "
                                       "median of 10 calls; frac of measured HBM peak by (N*s + S) / t"}
    compress_call()  # the headline stream again (its header differs: min / max recorded)

    # bytes the stage kernel writes: one staging slot per block,
    # [nnz | 0 | 64 coarse | B^3/8 mask bytes | nnz values]
    nblocks = (n // B) ** 3
    data0 = (cz.HEADER_BYTES + 8 * (nblocks + 1) + 15) // 16 * 16
    offs = out[cz.HEADER_BYTES:cz.HEADER_BYTES + 8 * nblocks].view(torch.int64)
    words = out[data0:data0 + (stream_len - data0 + 3) // 4 * 4].view(torch.int32)
    nnz_total = int(words[(offs // 4)].to(torch.int64).sum().item())
    stage1_written = nblocks * (8 + 64 * 4 + B ** 3 // 8) + 4 * nnz_total

    # end to end through the ABI with host buffers (pinned), copies included:
    # every step uploads the field, compresses, downloads the stream, decodes
    # and downloads the field.  Uploads, compressions, decodes, stream and
    # field downloads each run on a stream of their own, ordered by events;
    # two sets of device buffers let one field's upload overlap the previous
    # field's download (the link carries both directions at once).  The host
    # reads a step's stream length (and enqueues its downloads and decode)
    # once the next step's upload and compression are queued.  Every step's
    # copies are inside the timed region.
    e2e = None
    if not args.no_e2e:
        h_in = torch.from_numpy(field_np).pin_memory()
        depth = 2
        lanes = []
        for q in range(depth):
            lanes.append({
                "field": field if q == 0 else torch.empty_like(field),
                "out": out if q == 0 else torch.empty_like(out),
                "ws": ws if q == 0 else torch.empty_like(ws),
                "ws_d": torch.empty_like(ws),
                "nb": nb if q == 0 else torch.empty_like(nb),
                "rec": rec if q == 0 else torch.empty_like(rec),
                "h_out": torch.empty_like(h_in).pin_memory(),
                "h_stream": torch.empty(cap, dtype=torch.uint8).pin_memory(),
                "h_nb": torch.empty(1, dtype=torch.int64).pin_memory(),
                # the lane's buffers: field consumed, stream downloaded and
                # decoded, decoded field downloaded
                "ev_comp": torch.cuda.Event(), "ev_sdown": torch.cuda.Event(), "ev_dec": torch.cuda.Event(),
                "ev_fdown": torch.cuda.Event(),
            })
        s_up, s_c, s_d, s_sd, s_fd = (torch.cuda.Stream(dev) for _ in range(5))
        for L in lanes:
            for e_ in (L["ev_comp"], L["ev_sdown"], L["ev_dec"], L["ev_fdown"]):
                e_.record(s_c)
        torch.cuda.synchronize()
        copied_in = copied_out = 0

        def e2e_front(i):
            """Upload and compress field i (its lane's buffers once free)."""
            L = lanes[i % depth]
            ev_up = torch.cuda.Event()
            with torch.cuda.stream(s_up):
                s_up.wait_event(L["ev_comp"])  # the lane's previous field is consumed
                L["field"].copy_(h_in, non_blocking=True)
                ev_up.record(s_up)
            for e_ in (ev_up, L["ev_sdown"], L["ev_dec"]):  # the lane's previous stream is read
                s_c.wait_event(e_)
            r = cz.cz_compress(p, L["field"].data_ptr(), L["out"].data_ptr(), cap, L["nb"].data_ptr(),
                               L["ws"].data_ptr(), L["ws"].numel(), s_c.cuda_stream)
            if r != cz.OK:
                raise cz.CzError(r, "cz_compress")
            with torch.cuda.stream(s_c):
                L["h_nb"].copy_(L["nb"], non_blocking=True)
                L["ev_comp"].record(s_c)

        def e2e_back(i):
            """Download stream i, decode it and download the field."""
            nonlocal copied_in, copied_out
            L = lanes[i % depth]
            L["ev_comp"].synchronize()
            ln = int(L["h_nb"].item())
            with torch.cuda.stream(s_sd):
                s_sd.wait_event(L["ev_comp"])
                L["h_stream"][:ln].copy_(L["out"][:ln], non_blocking=True)
                L["ev_sdown"].record(s_sd)
            s_d.wait_event(L["ev_comp"])
            s_d.wait_event(L["ev_fdown"])  # the lane's previous field is downloaded
            r = cz.lib().cz_decompress(L["out"].data_ptr(), ln, hdr_c, L["rec"].data_ptr(), nbytes_field,
                                       L["ws_d"].data_ptr(), L["ws_d"].numel(), s_d.cuda_stream)
            if r != cz.OK:
                raise cz.CzError(r, "cz_decompress")
            L["ev_dec"].record(s_d)
            with torch.cuda.stream(s_fd):
                s_fd.wait_event(L["ev_dec"])
                L["h_out"].copy_(L["rec"], non_blocking=True)
                L["ev_fdown"].record(s_fd)
            copied_in = nbytes_field
            copied_out = 8 + ln + nbytes_field

        def e2e_run(steps):
            for i in range(steps):
                e2e_front(i)
                if i > 0:
                    e2e_back(i - 1)
            e2e_back(steps - 1)

        e2e_run(depth)
        torch.cuda.synchronize()
        reps = max(4, min(args.steps, 16))
        t0 = time.perf_counter()
        e2e_run(reps)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / reps
        for L in lanes:
            for w_ in (L["ws"], L["ws_d"]):
                st_ = cz.cz_status(w_.data_ptr(), s_c.cuda_stream)
                if st_ != cz.OK:
                    raise cz.CzError(st_, "device status after the end-to-end steps")
        if not torch.equal(lanes[0]["h_out"], lanes[1]["h_out"]):
            raise RuntimeError("end-to-end: the two lanes decoded different fields")
        e2e = {"value": world * nbytes_field / e2e_s / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": copied_in, "d2h_bytes_per_step": copied_out,
               "fields_in_flight": depth, "steps": reps}
        # the host link as plain cudaMemcpyAsync calls see it (one 4 GiB
        # copy at a time, pinned host memory), the bound of the figure above
        lib.czi_link_probe.argtypes = [cz.C.c_void_p, cz.C.c_void_p, cz.C.c_size_t, cz.C.c_int, cz.C.c_int,
                                       cz.C.c_void_p, cz.C.POINTER(cz.C.c_float)]
        lib.czi_link_probe.restype = cz.C.c_int
        link = {}
        L1 = lanes[1]
        for name, hb, db, dr in (("h2d_gbs", h_in, L1["field"], 0), ("d2h_gbs", L1["h_out"], L1["rec"], 1)):
            msv = cz.C.c_float()
            if lib.czi_link_probe(hb.data_ptr(), db.data_ptr(), nbytes_field, 3, dr, s, cz.C.byref(msv)) == cz.OK:
                link[name] = 3 * nbytes_field / (msv.value * 1e-3) / 1e9
        link["how"] = "3 x cudaMemcpyAsync of the 4 GiB field each way, pinned host buffer, CUDA events"
        # both directions at once (an upload and a download of 4 GiB on two
        # streams, as in the end-to-end steps): the bound of a step that
        # uploads one field while it downloads another
        cur = torch.cuda.current_stream(dev)
        sa, sb = s_fd, s_up
        both = []
        for _ in range(3):
            e0, ea, eb, e1 = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            e0.record(cur)
            sa.wait_event(e0)
            sb.wait_event(e0)
            with torch.cuda.stream(sa):
                lanes[0]["h_out"].copy_(lanes[0]["rec"], non_blocking=True)
                ea.record(sa)
            with torch.cuda.stream(sb):
                lanes[1]["field"].copy_(h_in, non_blocking=True)
                eb.record(sb)
            cur.wait_event(ea)
            cur.wait_event(eb)
            e1.record(cur)
            torch.cuda.synchronize()
            both.append(e0.elapsed_time(e1))
        link["both_directions_gbs"] = 2 * nbytes_field / (statistics.median(both) * 1e-3) / 1e9
        link["both_how"] = ("a 4 GiB upload and a 4 GiB download on two streams at once (bytes of both / time), "
                            "median of 3")
        e2e["host_link"] = link
        del lanes

    # other kinds (context: the headline is per kind), and bit zeroing
    # Z4 / Z8 of the kept details for the headline kind (Sec. 3, Exp. 2)
    def measure(pk, ws_=None):
        ws_ = ws if ws_ is None else ws_
        r = cz.cz_compress(pk, field.data_ptr(), out.data_ptr(), cap, nb.data_ptr(),
                           ws_.data_ptr(), ws_.numel(), s)
        assert r == cz.OK
        st_ = cz.cz_status(ws_.data_ptr(), s)
        if st_ != cz.OK:
            raise cz.CzError(st_, "compress (device)")
        ln = int(nb.item())
        hb = cz.C.create_string_buffer(out[:cz.HEADER_BYTES].cpu().numpy().tobytes(), 128)

        def kdec():
            r = cz.lib().cz_decompress(out.data_ptr(), ln, hb, rec.data_ptr(), nbytes_field,
                                       ws_.data_ptr(), ws_.numel(), s)
            assert r == cz.OK
        reps = 5
        ce = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a_, b_, c_ in ce:
            a_.record(stream)
            cz.cz_compress(pk, field.data_ptr(), out.data_ptr(), cap, nb.data_ptr(),
                           ws_.data_ptr(), ws_.numel(), s)
            b_.record(stream)
            kdec()
            c_.record(stream)
        torch.cuda.synchronize()
        cm = statistics.median(a_.elapsed_time(b_) for a_, b_, _ in ce)
        dm = statistics.median(b_.elapsed_time(c_) for _, b_, c_ in ce)
        d = rec.double() - field.double()
        mse_k = float((d * d).mean().item())
        del d
        return {"compress_gbs": nbytes_field / cm / 1e6, "decompress_gbs": nbytes_field / dm / 1e6,
                "cr": nbytes_field / ln,
                "psnr_db": 20 * math.log10((fmax - fmin) / (2 * math.sqrt(mse_k))) if mse_k > 0 else None}

    per_kind = {}
    bit_zeroing = block_sizes = aggregate = None
    if not args.headline_only:
        for kname, kk in cz.KINDS.items():
            per_kind[kname] = measure(cz.params_for(tuple(field.shape), False, B, kk, args.eps, cz.EPS_REL, True,
                                                    -1.0))
        bit_zeroing = {"kind": args.kind, "eps": args.eps}
        for z in (0, 4, 8):
            bit_zeroing[f"z{z}"] = measure(cz.params_for(tuple(field.shape), False, B, kind, args.eps, cz.EPS_REL,
                                                         True, -1.0, zero_bits=z))
        # block-size study (Sec. 3, Exp. 3): 8^3 / 16^3 / 32^3 / 64^3 blocks of the same field
        block_sizes = {"kind": args.kind, "eps": args.eps}
        for bb in (8, 16, 32, 64):
            pb = cz.params_for(tuple(field.shape), False, bb, kind, args.eps, cz.EPS_REL, True, -1.0)
            need = max(cz.cz_workspace_size(pb), ws.numel())
            ws_b = ws if need == ws.numel() else torch.empty(need, dtype=torch.uint8, device=dev)
            block_sizes[f"b{bb}"] = measure(pb, ws_b)
            del ws_b
        torch.cuda.empty_cache()
        # aggregate chunks (Sec. 3, Exp. 2 and 3): G consecutive blocks per
        # stage-2 chunk, against one chunk per block of the same edge
        aggregate = {"kind": args.kind, "eps": args.eps}
        for bb, gs in ((B, (4, 8)), (16, (16,)), (8, (16,))):
            for g in gs:
                pg = cz.params_for(tuple(field.shape), False, bb, kind, args.eps, cz.EPS_REL, True, -1.0, group=g)
                need = max(cz.cz_workspace_size(pg), ws.numel())
                ws_g = ws if need == ws.numel() else torch.empty(need, dtype=torch.uint8, device=dev)
                res = measure(pg, ws_g)
                res["cr_gain"] = res["cr"] / block_sizes[f"b{bb}"]["cr"] - 1
                aggregate[f"b{bb}_g{g}"] = res
                del ws_g
        torch.cuda.empty_cache()

    # random access with and without the decoded-block cache, on the
    # headline stream (compressed again: the studies above reused `out`)
    random_access = None
    if not args.headline_only and rank == 0:
        from paper_1903_07761_gb300 import workloads
        compress_call()
        ra_len = int(nb.item())
        random_access = workloads.random_access(out[:ra_len], ra_len, header)

    # batched fields and the served request stream (rank 0, one GPU)
    batched_res = served_res = fp64_res = config1_res = None
    if rank == 0 and world == 1:
        from paper_1903_07761_gb300 import workloads
        del rec
        torch.cuda.empty_cache()
        if not args.no_batch:
            batched_res = workloads.batched()
            torch.cuda.empty_cache()
        if not args.no_serve:
            # the full request-rate sweep of the served workload: 2000
            # requests at each of 100 ... 5000 per second
            served_res = workloads.served(rates=(100.0, 200.0, 500.0, 1000.0, 2000.0, 5000.0), n=2000)
            torch.cuda.empty_cache()
        if not args.no_fp64:
            fp64_res = workloads.fp64()
            torch.cuda.empty_cache()
        if not args.no_config1:
            config1_res = {"gpu": workloads.config1()}
            torch.cuda.empty_cache()

    # reductions over ranks (max time)
    if world > 1:
        total_ms, comp_ms, dec_ms, stage1_ms, dec2_ms, range_ms = rank_max(
            [total_ms, comp_ms, dec_ms, stage1_ms, dec2_ms, range_ms], dev)
    ms_per_step = total_ms / args.steps
    value = replica_throughput(world, nbytes_field, ms_per_step)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        slabs = max(1, args.cpu_slabs)
        byts, secs = cpu_oracle_run(field_np, B, kind, args.eps, slabs, fmax - fmin)
        cpu = {"value": byts / secs / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"compress+decompress of the first {min(slabs, n // B)} of the {n // B} z-slabs of {B} cells "
                         f"({byts / 2**20:.0f} MiB, {slabs * (n // B) ** 2} blocks) of the same "
                         f"field, threshold from the full range, single thread, {secs:.1f} s"}
        # context: the same oracle on every host core (independent tasks)
        try:
            aslabs = min(slabs, 8)
            ab, asecs, acores = cpu_oracle_all_cores(field_np, B, kind, args.eps, aslabs, fmax - fmin)
            cpu["all_cores"] = {"value": ab / asecs / 1e9, "unit": UNIT, "cores": acores,
                                "sample": f"the first {aslabs} z-slab(s) ({ab / 2**20:.0f} MiB) as "
                                          f"independent tasks on {acores} worker processes, {asecs:.2f} s"}
        except Exception as exc:  # context only: report, do not fail the run
            cpu["all_cores"] = {"unavailable": f"{type(exc).__name__}: {exc}"[:200]}
        # the oracle on the small field and on the bubble-cloud sweep (context)
        if config1_res is not None:
            try:
                config1_res["oracle"] = oracle_sweep_timing()
            except Exception as exc:
                config1_res["oracle"] = {"unavailable": f"{type(exc).__name__}: {exc}"[:200]}

    peak, peak_src = measured_peaks()
    # the major kernels' algorithmic bytes per launch, by the method's own
    # traffic (what compression and decompression must move): the stage
    # kernel reads the field and the compressed data is written (N*s + S);
    # the decode kernel reads the compressed data and writes the field
    # (S + N*s).  With the range computed, the stage kernel also merges the
    # field's min / max itself (speculative thresholds), after a min / max
    # pass over a subsample (every 4th row of every 4th z-plane: about
    # N*s / 16).  Stage-1 payloads in the workspace (S1, re-read by separate
    # stage-2 passes) are not counted.  `roofline` describes the kernel with
    # the largest time share, the others follow in `roofline_kernels`.
    sample_bytes = ((n + 3) // 4) * ((n + 3) // 4) * n * 4
    kernels = {
        "k_decompress2": (dec2_ms, nbytes_field + stream_len,
                          "k_decompress2 (payload scatter, inverse transform, TMA store of the tile)"),
        "k_stage1": (stage1_ms, nbytes_field + stream_len,
                     "k_stage1 (load, min/max, transform, threshold, mask, compaction)"),
        "k_minmax_sample": (range_ms, sample_bytes,
                            "k_minmax_sample (min/max of every 4th row of every 4th plane: a lower bound of the range)"),
    }

    def roof(name):
        ms, byts, what = kernels[name]
        ach = byts / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "kernel": what, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "peak_source": f"{peak_src} hbm_gbs (burst copy)",
                "traffic": traffic_per_launch(f"{name}_f32_b{B}_{args.kind}", nblocks),
                "algorithmic_bytes": byts, "kernel_ms": ms}

    dominant = max(kernels, key=lambda k: kernels[k][0])
    # k_minmax_sample, k_stage1, 2 x k_stage2 (small / large payloads),
    # k_stage2_refine, k_place, k_copy, 2 x k_unstage, k_decompress2
    launches_per_step = 10
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded bubble-cloud pressure field; paper datasets unavailable)",
        "config": workload_config(n, B, args.kind, world),
        "compress_gbs": nbytes_field / comp_ms / 1e6, "decompress_gbs": nbytes_field / dec_ms / 1e6,
        "compress_ms": comp_ms, "decompress_ms": dec_ms,
        "cr": nbytes_field / stream_len, "psnr_db": psnr, "linf_over_t": linf / (args.eps * (fmax - fmin)),
        "roofline": roof(dominant),
        "roofline_kernels": {k: roof(k) for k in kernels if k != dominant},
        "stage_ms": {"a0_minmax_sample": range_ms, "k_stage1": stage1_ms, "k_stage2": stage2_ms,
                     "k_place+k_copy": place_ms, "k_unstage": unstage_ms, "k_decompress2": dec2_ms},
        "compress_hbm_frac": (nbytes_field + stream_len) / (comp_ms * 1e-3) / 1e9 / peak,
        "stage1_bytes_written": stage1_written,
        "compress_range_supplied": compress_range_supplied,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "per_kind": per_kind,
        "bit_zeroing": bit_zeroing,
        "aggregate_chunks": aggregate,
        "block_sizes": block_sizes,
        "random_access": random_access,
        "batched": batched_res,
        "served": served_res,
        "fp64": fp64_res,
        "config1": config1_res,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    # the oracle and the input generator only (nothing of the CUDA library)
    kind = {"w4": 0, "w4li": 1, "w3ai": 2}[args.kind]
    n, B = args.n, args.block
    field_np = make_field(n, seed=2000)
    rng = float(field_np.max()) - float(field_np.min())
    slabs = 1
    for _ in range(args.warmup):
        cpu_oracle_run(field_np, B, kind, args.eps, slabs, rng)
    times = []
    byts = 0
    for _ in range(args.steps):
        byts, secs = cpu_oracle_run(field_np, B, kind, args.eps, slabs, rng)
        times.append(secs)
    ms = 1e3 * sum(times) / len(times)
    value = byts / (ms * 1e-3) / 1e9
    sample = (f"compress+decompress of one z-slab of {B} cells ({byts / 2**20:.0f} MiB, "
              f"{(n // B) ** 2} blocks) of the {n}^3 field per step, single thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(n, B, args.kind, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def build_parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="cz", choices=["cz", "reference"])
    ap.add_argument("--kind", default="w3ai", choices=["w4", "w4li", "w3ai"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--block", type=int, default=32)
    ap.add_argument("--eps", type=float, default=1e-3)
    ap.add_argument("--cpu-slabs", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--headline-only", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-fields comparison")
    ap.add_argument("--no-serve", action="store_true", help="skip the served-requests comparison")
    ap.add_argument("--no-fp64", action="store_true", help="skip the 768^3 FP64 case")
    ap.add_argument("--no-config1", action="store_true", help="skip the 512^3 bubble-cloud sweep")
    return ap


def main():
    args = build_parser().parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
