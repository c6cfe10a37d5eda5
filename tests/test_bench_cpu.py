"""The benchmark's reference arm (the FP64 oracle on host cores) runs without
a GPU; its JSON line carries the keys the measurement contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run("--impl", "reference", "--workload", "tiny", "--steps", "2", "--warmup", "3")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"].startswith("tiny")


def test_warmup_floor():
    d = _run("--impl", "reference", "--workload", "tiny", "--steps", "1", "--warmup", "1")
    assert d["warmup"] >= 3


def test_threaded_oracle_timing_covers_the_sample():
    """The all-cores CPU baseline runs the unchanged oracle on interleaved row
    shares; the shares partition the sample exactly."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    P, _ = bench.load_workload("tiny")
    rows, nnz, stride = bench.oracle_sample_rows(P, 0, 20_000)
    shares = [rows[t::3] for t in range(3)]
    assert np.array_equal(np.sort(np.concatenate(shares)), rows)
    assert bench.time_oracle_step_threads(P, rows, 3) > 0
    assert bench.host_cores() >= 1
