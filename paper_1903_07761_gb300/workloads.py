"""Batched and served workloads on the GPU, measured against plain launches.

* batched(): 64 fields with edge lengths log-uniform on [64, 384] (each axis
  drawn on its own, rounded to a multiple of 32), half FP32 (32^3 blocks) and
  half FP64 (16^3 blocks), eps drawn from {1e-2, 1e-3, 1e-4} per field,
  W3ai, content from the bubble-cloud pressure recipe; compressed by one
  tuned cz_compress_batch call replayed from a CUDA graph, against the 64
  cz_compress calls one after another.  The streams are identical, so the
  PSNRs are equal.
* served(): a Poisson stream of compress and decompress requests (1:1) of
  cubic fields with edges log-uniform on [32, 512] (rounded to 32), 70 % FP32
  and 30 % FP64, eps in {1e-3, 1e-4}, through the request server under an
  HBM budget, against one-at-a-time plain launches on the same trace.

* config1(): the bubble-cloud sweep -- gas fraction, density and pressure
  of one 200-bubble cloud on a 512^3 domain (FP32, 32^3 blocks), every
  kind at eps in {1e-2, 1e-3, 1e-4, 1e-5}: compression factor, PSNR, the
  largest error over the threshold, and compress / decompress GB/s (the
  paper's wavelet-type experiment, Sec. 3 Exp. 1, on synthetic fields).

All return plain dicts for the benchmark line.  Inputs are synthetic
(seeded); see inputs/czgen.c.
"""
from __future__ import annotations

import ctypes as C
import json
import math
import time

import numpy as np

from . import cz, inputs


def _loguniform_edge(rng, lo, hi):
    e = math.exp(rng.uniform(math.log(lo), math.log(hi)))
    return int(max(lo, min(hi, round(e / 32) * 32)))


# ------------------------------------------------------------------ batched
def batched(nfields: int = 64, reps: int = 10, seed: int = 3000, nbubbles: int = 200):
    import torch
    rng = np.random.default_rng(seed)
    fields, params, bytes_total = [], [], 0
    for i in range(nfields):
        f64 = i % 2 == 1
        dims = tuple(_loguniform_edge(rng, 64, 384) for _ in range(3))
        eps = float(rng.choice([1e-2, 1e-3, 1e-4]))
        f = inputs.field(inputs.P, dims, np.float64 if f64 else np.float32, seed=seed + i,
                         nbubbles=nbubbles)
        t = torch.from_numpy(f).cuda()
        fields.append(t)
        B = 16 if f64 else 32
        params.append(cz.params_for(tuple(t.shape), f64, B, "w3ai", eps))
        bytes_total += t.numel() * t.element_size()
    caps = [cz.cz_compress_bound(p) for p in params]
    outs = [torch.zeros(c, dtype=torch.uint8, device="cuda") for c in caps]
    nbytes = torch.zeros(nfields, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream

    # plain: one cz_compress per field, one after another (own workspace sized
    # for the largest field)
    ws_plain = torch.empty(max(cz.cz_workspace_size(p) for p in params), dtype=torch.uint8, device="cuda")
    one = torch.zeros(1, dtype=torch.int64, device="cuda")

    def plain():
        for p, t, o, c in zip(params, fields, outs, caps):
            r = cz.cz_compress(p, t.data_ptr(), o.data_ptr(), c, one.data_ptr(), ws_plain.data_ptr(),
                               ws_plain.numel(), s)
            assert r == cz.OK

    plain()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        plain()
    e1.record()
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1) / reps
    # streams of the plain path, to compare with the batched ones
    plain_streams = []
    for p, t, o, c in zip(params, fields, outs, caps):
        r = cz.cz_compress(p, t.data_ptr(), o.data_ptr(), c, one.data_ptr(), ws_plain.data_ptr(),
                           ws_plain.numel(), s)
        assert r == cz.OK
        torch.cuda.synchronize()
        plain_streams.append(bytes(o[:int(one.item())].cpu().numpy()))
    del ws_plain

    # batched: one call captured in a CUDA graph and replayed, first with the
    # default knobs, then after the tuner has chosen them for each group
    ws = torch.empty(cz.cz_batch_workspace_size(params), dtype=torch.uint8, device="cuda")
    b = cz.BatchArgs(params, [t.data_ptr() for t in fields], [o.data_ptr() for o in outs], caps)

    def graph_ms():
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            assert cz.cz_compress_batch(b, nbytes.data_ptr(), ws.data_ptr(), ws.numel(), side.cuda_stream) == cz.OK
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            assert cz.cz_compress_batch(b, nbytes.data_ptr(), ws.data_ptr(), ws.numel(),
                                        torch.cuda.current_stream().cuda_stream) == cz.OK
        g.replay()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    untuned_ms = graph_ms()
    t0 = time.perf_counter()
    assert cz.cz_batch_tune(b, nbytes.data_ptr(), ws.data_ptr(), ws.numel(), s, 3) == cz.OK
    tune_s = time.perf_counter() - t0
    batch_ms = graph_ms()
    n = C.c_size_t()
    assert cz.lib().cz_batch_knobs_export(None, 0, C.byref(n)) == cz.OK
    buf = C.create_string_buffer(n.value)
    assert cz.lib().cz_batch_knobs_export(C.cast(buf, C.c_void_p), n.value, C.byref(n)) == cz.OK
    knobs = json.loads(buf.value.decode())["entries"]
    lens = nbytes.cpu().tolist()
    same = all(bytes(o[:n].cpu().numpy()) == ps for o, n, ps in zip(outs, lens, plain_streams))
    stream_bytes = sum(lens)
    # PSNR of a few fields (identical streams give identical PSNR on both paths)
    ps = []
    for i in range(0, nfields, 16):
        rec = cz.decompress(outs[i], nbytes=lens[i])
        d = rec.double() - fields[i].double()
        mse = float((d * d).mean().item())
        rg = float(fields[i].max().item() - fields[i].min().item())
        ps.append(20 * math.log10(rg / (2 * math.sqrt(mse))) if mse > 0 else float("inf"))
    return {
        "workload": f"{nfields} fields, edges log-uniform [64,384] step 32, FP32 32^3 / FP64 16^3 blocks, "
                    f"eps in {{1e-2,1e-3,1e-4}}, W3ai, range computed",
        "field_bytes": bytes_total, "stream_bytes": stream_bytes,
        "plain_ms": plain_ms, "plain_gbs": bytes_total / plain_ms / 1e6,
        "batched_ms": batch_ms, "batched_gbs": bytes_total / batch_ms / 1e6,
        "speedup": plain_ms / batch_ms, "streams_identical": same,
        "untuned_batched_ms": untuned_ms, "tuned_over_untuned": untuned_ms / batch_ms, "tune_s": tune_s,
        "tuned_knobs": knobs,
        "knobs": "per group: slab = stage kernel with the block in global scratch (FP32 32^3 only) instead of "
                 "in registers; s1_balanced = fewest stage CTAs with the same rounds; s2_div = stage-2 CTAs "
                 "/ resident slots; place_tile = chunks per look-back tile",
        "psnr_db_sample": ps, "graph": True,
    }


# ------------------------------------------------------------------ served
class _Pool:
    """Device fields and streams of every size class of the served trace."""

    def __init__(self, seed: int, nbubbles: int, max_edge: int):
        import torch
        self.fields, self.streams = {}, {}
        base = {}
        for f64 in (False, True):
            dt = np.float64 if f64 else np.float32
            base[f64] = torch.from_numpy(inputs.field(inputs.P, (max_edge,) * 3, dt, seed=seed + int(f64),
                                                      nbubbles=nbubbles)).cuda()
        for e in range(32, max_edge + 1, 32):
            for f64 in (False, True):
                self.fields[(e, f64)] = base[f64][:e, :e, :e].contiguous()
        self.base = base

    def stream_of(self, e, f64, eps, kind):
        key = (e, f64, eps, kind)
        if key not in self.streams:
            out, nb = cz.compress(self.fields[(e, f64)], block=32, kind=kind, eps=eps)
            n = int(nb.item())
            self.streams[key] = (out[:n].clone(), n, out[:cz.HEADER_BYTES].cpu().numpy().tobytes())
        return self.streams[key]


def _trace(rate: float, n: int, seed: int, max_edge: int):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    reqs = []
    for i in range(n):
        e = _loguniform_edge(rng, 32, max_edge)
        f64 = rng.random() < 0.3
        eps = float(rng.choice([1e-3, 1e-4]))
        op = cz.OP_COMPRESS if i % 2 == 0 else cz.OP_DECOMPRESS
        reqs.append((float(t[i]), op, e, f64, eps))
    return reqs


def served(rates=(1000.0, 5000.0), n: int = 400, budget_gb: float = 40.0, streams: int = 4,
           seed: int = 4000, nbubbles: int = 200, max_edge: int = 512, kind: str = "w3ai"):
    import torch
    pool = _Pool(seed, nbubbles, max_edge)
    # output buffers: a small ring per size class and op (requests of one
    # class that overlap may share a buffer: their outputs are not read)
    ring = 2
    outs = {}

    def out_for(op, e, f64, i):
        key = (op, e, f64, i % ring)
        if key not in outs:
            p = cz.params_for((e, e, e), f64, 32, kind, 1e-3)
            nbytes = cz.cz_compress_bound(p) if op == cz.OP_COMPRESS else e ** 3 * (8 if f64 else 4)
            outs[key] = (torch.empty(nbytes, dtype=torch.uint8, device="cuda"),
                         torch.zeros(1, dtype=torch.int64, device="cuda"))
        return outs[key]

    # load every kernel the trace uses once before any clock starts (CUDA
    # loads a kernel's module at its first launch): plain and batched
    # compress and decompress, FP32 and FP64 32^3 blocks, and the same
    # through a server
    warm = []
    for f64 in (False, True):
        B = 32
        f = pool.fields[(32, f64)]
        st, nb = cz.compress(f, block=B, kind=kind, eps=1e-3)
        cz.decompress(st, nbytes=int(nb.item()))
        cz.compress_batch([f, f], block=B, kind=kind, eps=1e-3)
        warm += [(0.0, cz.OP_COMPRESS, 32, f64, 1e-3), (0.0, cz.OP_DECOMPRESS, 32, f64, 1e-3)] * 2
    with cz.Server(int(budget_gb * (1 << 30)), streams) as srv:
        tks = []
        for i, (_, op, e, f64, eps) in enumerate(warm):
            o, nb = out_for(op, e, f64, i)
            if op == cz.OP_COMPRESS:
                p = cz.params_for((e, e, e), f64, 32, kind, eps)
                tks.append(srv.submit_compress(p, pool.fields[(e, f64)].data_ptr(), o.data_ptr(), o.numel(),
                                               nb.data_ptr()))
            else:
                sd, sn, hdr = pool.stream_of(e, f64, eps, kind)
                tks.append(srv.submit_decompress(sd.data_ptr(), sn, hdr, o.data_ptr(), o.numel()))
        for tk in tks:
            assert srv.wait(tk)[0] == cz.OK
    torch.cuda.synchronize()

    results = []
    for rate in rates:
        reqs = _trace(rate, n, seed + int(rate), max_edge)
        for _, op, e, f64, eps in reqs:  # decompress inputs, made before the clock starts
            if op == cz.OP_DECOMPRESS:
                pool.stream_of(e, f64, eps, kind)
        torch.cuda.synchronize()
        nbytes_total = sum(e ** 3 * (8 if f64 else 4) for _, _, e, f64, _ in reqs)

        # ---- through the server
        lat = []
        with cz.Server(int(budget_gb * (1 << 30)), streams) as srv:
            tickets = []
            t0 = time.perf_counter()
            for i, (ta, op, e, f64, eps) in enumerate(reqs):
                while time.perf_counter() - t0 < ta:
                    pass
                o, nb = out_for(op, e, f64, i)
                if op == cz.OP_COMPRESS:
                    p = cz.params_for((e, e, e), f64, 32, kind, eps)
                    tk = srv.submit_compress(p, pool.fields[(e, f64)].data_ptr(), o.data_ptr(), o.numel(),
                                             nb.data_ptr())
                else:
                    sd, sn, hdr = pool.stream_of(e, f64, eps, kind)
                    tk = srv.submit_decompress(sd.data_ptr(), sn, hdr, o.data_ptr(), o.numel())
                tickets.append(tk)
            for tk in tickets:
                res, ms = srv.wait(tk)
                assert res == cz.OK, res
                lat.append(ms)
            wall = time.perf_counter() - t0
        srv_gbs = nbytes_total / wall / 1e9

        # ---- one at a time, plain launches, same trace
        s = torch.cuda.current_stream().cuda_stream
        ws = torch.empty(max(cz.cz_workspace_size(cz.params_for((e, e, e), f64, 32, kind, eps))
                             for _, _, e, f64, eps in reqs), dtype=torch.uint8, device="cuda")
        plat = []
        t0 = time.perf_counter()
        for i, (ta, op, e, f64, eps) in enumerate(reqs):
            while time.perf_counter() - t0 < ta:
                pass
            o, nb = out_for(op, e, f64, i)
            if op == cz.OP_COMPRESS:
                p = cz.params_for((e, e, e), f64, 32, kind, eps)
                r = cz.cz_compress(p, pool.fields[(e, f64)].data_ptr(), o.data_ptr(), o.numel(), nb.data_ptr(),
                                   ws.data_ptr(), ws.numel(), s)
            else:
                sd, sn, hdr = pool.stream_of(e, f64, eps, kind)
                r = cz.cz_decompress(sd.data_ptr(), sn, hdr, o.data_ptr(), o.numel(), ws.data_ptr(), ws.numel(), s)
            assert r == cz.OK
            torch.cuda.current_stream().synchronize()
            plat.append((time.perf_counter() - t0 - ta) * 1e3)
        pwall = time.perf_counter() - t0
        del ws
        results.append({
            "rate_per_s": rate, "requests": n,
            "server": {"gbs": srv_gbs, "p50_ms": float(np.percentile(lat, 50)),
                       "p99_ms": float(np.percentile(lat, 99)), "wall_s": wall},
            "plain": {"gbs": nbytes_total / pwall / 1e9, "p50_ms": float(np.percentile(plat, 50)),
                      "p99_ms": float(np.percentile(plat, 99)), "wall_s": pwall},
        })
    return {
        "workload": f"Poisson compress/decompress 1:1, cubic edges log-uniform [32,{max_edge}] step 32, "
                    f"70% FP32 / 30% FP64, 32^3 blocks, eps in {{1e-3,1e-4}}, {kind}, "
                    f"budget {budget_gb:g} GB, {streams} streams",
        "runs": results,
    }


# ------------------------------------------------------------------ random access
def random_access(stream_t, nbytes: int, header: bytes, steps: int = 200, capacity: int = 64, seed: int = 5000,
                  radius: int = 1):
    """Analysis-style random access (Sec. 2.3, Data decompression): a probe
    point walks through the block grid, one block per step along a random
    axis, and each step fetches the (2 radius + 1)^3 blocks around it
    (clamped at the faces).  Consecutive neighbourhoods share most blocks,
    which the decoded-block cache serves without decoding; the comparison
    decodes every requested block with cz_decompress_blocks."""
    import torch
    p, _ = cz.cz_read_header(header)
    B = p.block
    nbx, nby, nbz = p.nx // B, p.ny // B, p.nz // B
    rng = np.random.default_rng(seed)
    pos = np.array([nbx // 2, nby // 2, nbz // 2])
    reqs = []
    for _ in range(steps):
        ax = int(rng.integers(0, 3))
        pos[ax] = min(max(pos[ax] + int(rng.choice([-1, 1])), 0), (nbx, nby, nbz)[ax] - 1)
        ids = []
        rr = range(-radius, radius + 1)
        for dz in rr:
            for dy in rr:
                for dx in rr:
                    x = min(max(pos[0] + dx, 0), nbx - 1)
                    y = min(max(pos[1] + dy, 0), nby - 1)
                    z = min(max(pos[2] + dz, 0), nbz - 1)
                    ids.append(int((z * nby + y) * nbx + x))
        reqs.append(ids)
    dev_ids = [torch.tensor(r, dtype=torch.int32, device=stream_t.device) for r in reqs]
    nreq1 = (2 * radius + 1) ** 3
    out = torch.empty((nreq1, B, B, B), dtype=torch.float64 if p.dtype == cz.F64 else torch.float32,
                      device=stream_t.device)
    ws = cz.Workspace(stream_t.device)
    # warm-up of both paths (kernel loading), then the timed walks
    cz.decompress_blocks(stream_t, dev_ids[0], nbytes, header, out=out, ws=ws)
    cache = cz.Cache(capacity, B, f64=p.dtype == cz.F64)
    cache.fetch(stream_t, reqs[0], nbytes, header, out=out, ws=ws)
    cache.clear()
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record()
    for d in dev_ids:
        cz.decompress_blocks(stream_t, d, nbytes, header, out=out, ws=ws, check=False)
    e[1].record()
    hits = 0
    e[2].record()
    for r in reqs:
        hits += cache.fetch(stream_t, r, nbytes, header, out=out, ws=ws, check=False)[1]
    e[3].record()
    torch.cuda.synchronize()
    plain_ms, cache_ms = e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3])
    st = cz.cz_status(ws.buf.data_ptr(), torch.cuda.current_stream().cuda_stream)
    if st != cz.OK:
        raise cz.CzError(st, "random access (device)")
    held, _, decoded = cache.stats()
    cache.close()
    nreq = steps * nreq1
    return {
        "workload": f"probe walk of {steps} steps through the {nbx}x{nby}x{nbz} grid of {B}^3 "
                    f"{'FP64' if p.dtype == cz.F64 else 'FP32'} blocks, {nreq1} neighbouring blocks per step, "
                    f"cache of {capacity} tiles",
        "blocks_requested": nreq, "blocks_decoded_with_cache": decoded, "hit_rate": hits / nreq,
        "plain_ms_per_step": plain_ms / steps, "cache_ms_per_step": cache_ms / steps,
        "speedup": plain_ms / cache_ms,
    }


# ------------------------------------------------------------------ FP64
def _w3ai_fp64_ops_per_element(B: int, xy_run_time: bool = True) -> float:
    """FP64 instructions per element of the exact-build W3ai transform (one
    direction) over all levels and axes, counted from the kernels' steps.
    Forward, per pair: the average (add, mul), the predicted half-cell value
    and the detail (sub); inverse, per pair: the predicted value, its sum
    with the detail (add) and the second sample (mul, sub).  Compile-time
    rows (interior form one subtraction) take 6 operations per interior
    pair and 10 at the two boundary pairs of a line.  In the register-
    resident kernels the finest x- and y-steps use run-time stencils
    (xy_run_time): 8 operations per interior pair (two weight multiplies,
    add, multiply by 1/8, add) and 10 at the boundary pairs; the slab
    kernels of 32^3 FP64 blocks use compile-time rows on every line."""
    total, frac, n, level = 0.0, 1.0, B, 0
    while n >= 8:
        m = n // 2
        run_time = (m - 2) * 8 + 2 * 10
        compile_time = (m - 2) * 6 + 2 * 10
        if level == 0 and xy_run_time:
            lines = 2 * run_time + compile_time
        else:
            lines = 3 * compile_time
        total += frac * lines / n
        n //= 2
        frac /= 8
        level += 1
    return total


def _fp64_case(f, B: int, kind: str, eps: float, reps: int):
    """Compress / decompress times (ms) and stream bytes of field f."""
    import ctypes as C
    import torch
    nbytes = f.numel() * 8
    p = cz.params_for(tuple(f.shape), True, B, kind, eps)
    cap = cz.cz_compress_bound(p)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    ws = torch.empty(cz.cz_workspace_size(p), dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    rec = torch.empty_like(f)
    s = torch.cuda.current_stream().cuda_stream

    def comp():
        assert cz.cz_compress(p, f.data_ptr(), out.data_ptr(), cap, nb.data_ptr(), ws.data_ptr(), ws.numel(), s) == cz.OK

    comp()
    ln = int(nb.item())
    hdr = C.create_string_buffer(out[:cz.HEADER_BYTES].cpu().numpy().tobytes(), cz.HEADER_BYTES)

    def dec():
        assert cz.lib().cz_decompress(out.data_ptr(), ln, hdr, rec.data_ptr(), nbytes, ws.data_ptr(), ws.numel(), s) == cz.OK

    c_ms, d_ms = _timed(comp, reps), _timed(dec, reps)
    torch.cuda.synchronize()
    err = float((rec - f).abs().max())
    del out, ws, rec
    return c_ms, d_ms, ln, err


def _timed(fn, reps):
    import torch
    for _ in range(2):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def fp64(n: int = 768, kind: str = "w3ai", eps: float = 1e-3, reps: int = 10, seed: int = 2001):
    """The FP64 case: 768^3 density field in 16^3 blocks, and the same field
    in 32^3 blocks (the slab kernels).  GB300's FP64 rate is low enough that
    this path is bound by the FP64 pipe, not by HBM; the FP64 rate is
    measured here with a probe kernel (independent DFMA chains)."""
    import ctypes as C
    import torch
    f = torch.from_numpy(inputs.cavitation("rho", n, np.float64, seed=seed)).cuda()
    nbytes = f.numel() * 8
    s = torch.cuda.current_stream().cuda_stream
    # FP64 probe: DFMA instructions per second
    L = cz.lib()
    L.czi_fp64_probe.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
    L.czi_fp64_probe.restype = C.c_int
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    grid, thr, iters = sms * 8, 256, 4096

    def probe():
        assert L.czi_fp64_probe(grid, thr, iters, sink.data_ptr(), s) == cz.OK

    p_ms = _timed(probe, reps)
    dfma_per_s = grid * thr * iters * 8 / (p_ms * 1e-3)
    try:
        import json, os
        with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")) as fh:
            peaks = float(json.load(fh)["hbm_gbs"])
    except Exception:
        peaks = 6800.0

    def case(B):
        c_ms, d_ms, ln, err = _fp64_case(f, B, kind, eps, reps)
        dops = _w3ai_fp64_ops_per_element(B, xy_run_time=(B != 32))
        ops = dops + 1.0  # + the significance compare
        return {
            "compress_ms": c_ms, "decompress_ms": d_ms,
            "compress_gbs": nbytes / c_ms / 1e6, "decompress_gbs": nbytes / d_ms / 1e6,
            "cr": nbytes / ln, "linf": err,
            "hbm_frac_compress": (2 * nbytes + ln) / (c_ms * 1e-3) / 1e9 / peaks,
            "hbm_frac_decompress": (ln + nbytes) / (d_ms * 1e-3) / 1e9 / peaks,
            "fp64_ops_per_element": {"compress": ops, "decompress": dops},
            "fp64_pipe_frac_compress": ops * f.numel() / (c_ms * 1e-3) / dfma_per_s,
            "fp64_pipe_frac_decompress": dops * f.numel() / (d_ms * 1e-3) / dfma_per_s,
        }

    r = case(16)
    r32 = case(32)
    # random access on the 32^3 stream: decoding is FP64-bound here, so the
    # decoded-block cache saves time, not only work
    st32, nb32 = cz.compress(f, block=32, kind=kind, eps=eps)
    ln32 = int(nb32.item())
    ra = random_access(st32[:ln32], ln32, st32[:cz.HEADER_BYTES].cpu().numpy().tobytes(), steps=60,
                       capacity=512, radius=3)
    del st32
    torch.cuda.empty_cache()
    r.update({
        "workload": f"rho-field {n}^3 FP64, 16^3 blocks, {kind}, eps=1e-3*range, stage 2 on, range computed",
        "fp64_probe_dfma_per_s": dfma_per_s,
        "bound": "fp64 alu",
        "blocks_32": dict(r32, workload=f"the same field in 32^3 blocks (slab kernels: the block in global "
                                         f"memory, L2-resident)"),
        "random_access_32": ra,
    })
    return r


# ------------------------------------------------------------------ bubble-cloud sweep
def config1(n: int = 512, fields=("alpha", "rho", "p"), kinds=("w4", "w4li", "w3ai"),
            eps_list=(1e-2, 1e-3, 1e-4, 1e-5), reps: int = 3, seed: int = 1000, nbubbles: int = 200):
    """Every (field, kind, eps) of the sweep: the stream is made once, then
    compress and decompress are each timed `reps` times (median, CUDA
    events, range computed on the device as in the headline)."""
    import statistics

    import torch
    s = torch.cuda.current_stream().cuda_stream
    rows = []
    for fname in fields:
        f = torch.from_numpy(inputs.cavitation(fname, n, np.float32, seed=seed, nbubbles=nbubbles)).cuda()
        nbytes_field = f.numel() * 4
        fmin, fmax = float(f.min().item()), float(f.max().item())
        rng = fmax - fmin
        rec = torch.empty_like(f)
        for kind in kinds:
            for eps in eps_list:
                p = cz.params_for(tuple(f.shape), False, 32, kind, eps)
                cap = cz.cz_compress_bound(p)
                out = torch.empty(cap, dtype=torch.uint8, device="cuda")
                ws = torch.empty(cz.cz_workspace_size(p), dtype=torch.uint8, device="cuda")
                nb = torch.zeros(1, dtype=torch.int64, device="cuda")

                def comp():
                    r = cz.cz_compress(p, f.data_ptr(), out.data_ptr(), cap, nb.data_ptr(), ws.data_ptr(),
                                       ws.numel(), s)
                    assert r == cz.OK

                comp()
                assert cz.cz_status(ws.data_ptr(), s) == cz.OK
                ln = int(nb.item())
                hdr = out[:cz.HEADER_BYTES].cpu().numpy().tobytes()

                def dec():
                    r = cz.cz_decompress(out.data_ptr(), ln, hdr, rec.data_ptr(), nbytes_field, ws.data_ptr(),
                                         ws.numel(), s)
                    assert r == cz.OK

                tc, td = [], []
                for _ in range(reps):
                    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                    e0.record()
                    comp()
                    e1.record()
                    dec()
                    e2.record()
                    torch.cuda.synchronize()
                    tc.append(e0.elapsed_time(e1))
                    td.append(e1.elapsed_time(e2))
                assert cz.cz_status(ws.data_ptr(), s) == cz.OK
                d = rec.double() - f.double()
                mse = float((d * d).mean().item())
                linf = float(d.abs().max().item())
                del d
                cm, dm = statistics.median(tc), statistics.median(td)
                rows.append({
                    "field": fname, "kind": kind, "eps": eps, "cr": nbytes_field / ln,
                    "psnr_db": 20 * math.log10(rng / (2 * math.sqrt(mse))) if mse > 0 else None,
                    "linf_over_t": linf / (eps * rng) if rng > 0 else None,
                    "compress_gbs": nbytes_field / cm / 1e6, "decompress_gbs": nbytes_field / dm / 1e6,
                })
                del out, ws
        del f, rec
        torch.cuda.empty_cache()
    return {"workload": f"bubble cloud ({nbubbles} tanh-interface bubbles, seed {seed}) on {n}^3, FP32, "
                        f"32^3 blocks, fields {'/'.join(fields)}, stage 2 on, range computed; "
                        f"{reps} timed calls each (median)",
            "rows": rows}
