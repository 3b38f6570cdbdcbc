"""The JSON line of `bench.py` (CPU only): the reference arm (the oracle on the
host cores) prints one line with the keys of the measurement contract, and the
product arm, with no CUDA device, exits non-zero without printing a
measurement (no host fallback)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, timeout):
    return subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, capture_output=True, text=True,
                          timeout=timeout)


def _lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def test_reference_arm_line():
    p = _run(["--impl", "reference", "--steps", "1", "--warmup", "1"], timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = _lines(p.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["unit"] == "cells/s" and d["data"] == "synthetic"
    assert d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_product_arm_needs_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    p = _run(["--steps", "3", "--warmup", "3"], timeout=300)
    assert p.returncode != 0
    assert not [d for d in _lines(p.stdout) if "value" in d]


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"], cwd=ROOT,
                       capture_output=True, text=True, timeout=300, env=env)
    assert p.returncode == 0
    assert not _lines(p.stdout)


def test_step_byte_counts_follow_the_scope_table():
    """Floor = outputs + amplitudes once per batch; plan = floor + the pruned
    intermediates written and read once.  The 512^2 workload: 2 fields and 2
    count maps of 512^2 cells (4 MiB) + 1024^2 amplitudes / 64 realizations
    (64 KiB); plan + 1024 x 512 complex written and read (8 MiB).  The
    binary64 64^2 workload: 2 fields of 8 bytes (64 KiB) + 128^2 amplitudes of
    8 bytes / 16 realizations; plan + 128 x 64 complex of 16 bytes twice."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1406_6072_gb300 import workloads as W
    mib = float(1 << 20)
    wl = W.CONFIGS["cauchy2d_n512_f32"]
    floor, plan = bench.step_bytes(wl, wl.R)
    assert floor == 4 * (1 << 20) + 64 * 1024
    assert plan == floor + 8 * (1 << 20)
    wl = W.CONFIGS["gauss2d_n64_f64"]
    floor, plan = bench.step_bytes(wl, wl.R)
    assert floor == 2 * 64 * 64 * 8 + 128 * 128 * 8 / 16
    assert plan == floor + 2 * 128 * 64 * 16
    assert round(floor / mib, 2) == 0.07 and round(plan / mib, 2) == 0.32
