"""The benchmark's host-side parts, without a GPU: the reference arm (the
oracle on the host cores) prints one JSON line with the keys the benchmark
contract asks for, and the all-cores oracle run processes exactly its
sample."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "128",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] >= 3 and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_all_cores_oracle_run_covers_its_sample():
    sys.path.insert(0, ROOT)
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    sys.modules["bench"] = bench
    spec.loader.exec_module(bench)
    import oracle as O
    from paper_1903_07761_gb300 import inputs
    f = inputs.cavitation("p", 64, np.float32, seed=3)
    byts, secs, cores = bench.cpu_oracle_all_cores(f, 32, O.W3AI, 1e-3, 2, float(f.max() - f.min()))
    assert byts == f.nbytes and secs > 0 and cores >= 1


def test_profile_commands_run_committed_files_with_valid_flags():
    """Every profile summary gives the command that made it; each
    `python bench.py ...` there must still parse with the benchmark's
    options, and every file a command names must be in the repository."""
    import glob
    import importlib.util
    import shlex
    spec = importlib.util.spec_from_file_location("bench_for_profiles", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    parser = bench.build_parser()
    tracked = set(subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True,
                                 check=True).stdout.split())
    found = 0
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(path).read().replace("\\\n", " ")
        for line in text.splitlines():
            line = line.split("#")[0]
            if "python bench.py" not in line:
                continue
            args = shlex.split(line.split("python bench.py", 1)[1])
            parser.parse_args(args)  # exits on an unknown option
            found += 1
        for name in ("bench.py", "__graft_entry__.py"):
            if name in text:
                assert name in tracked
    assert found >= 3


def test_oracle_sweep_timing_reports_every_part():
    """The oracle timings beside the bubble-cloud sweep (single thread and
    all host cores), on a 64^3 cloud so that the test stays short."""
    sys.path.insert(0, ROOT)
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    sys.modules["bench"] = bench
    spec.loader.exec_module(bench)
    out = bench.oracle_sweep_timing(n1=64)
    assert out["cores_all"] >= 1
    for k in ("small_single", "small_all", "cloud_all"):
        assert out[k]["gbs"] > 0 and out[k]["cores"] >= 1
    assert set(out["cloud_single_p_eps1e-3"]["per_kind"]) == {"w4", "w4li", "w3ai"}
    assert "36 runs" in out["cloud_all"]["what"]
