"""bench.py's reference arm (the FP64 oracle on the host) prints one JSON line
with the keys the benchmark contract names; runs on CPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e")


def _run(*extra):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", *extra], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in KEYS:
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    return d


def test_reference_arm_hierarchical():
    d = _run("--workload", "hierarchical")
    assert d["unit"] == "windows/s" and d["config"]["workload"] == "hierarchical"


def test_reference_arm_precision_is_the_default():
    # the default workload; one query per step keeps the FP64 scan of 2,000,000 rows short
    d = _run("--ref-per-step", "1")
    assert d["unit"] == "queries/s" and d["config"]["workload"] == "precision"
    assert d["cpu_baseline"]["cores"] == 1 and d["config"]["units_per_step"] == 1


def test_default_workload_is_precision():
    sys.path.insert(0, ROOT)
    import bench
    src = open(os.path.join(ROOT, "bench.py")).read()
    assert 'ap.add_argument("--workload", default="precision"' in src
    assert bench.METRIC.startswith("queries/s")


@pytest.mark.parametrize("n,threads", [(3, 1), (5, 3)])
def test_oracle_thread_pool_matches_one_thread(n, threads):
    # the CPU baseline's worker threads return exactly what one thread returns
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    rng = np.random.default_rng(7)
    X = rng.standard_normal((3000, 16)).astype(np.float32)
    Q = rng.standard_normal((n, 16)).astype(np.float32)
    i1, d1, _ = bench.oracle_topk_threads(Q, X, 5, 1)
    it, dt, _ = bench.oracle_topk_threads(Q, X, 5, threads)
    assert np.array_equal(i1, it) and np.array_equal(d1, dt)
