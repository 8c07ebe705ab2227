"""bench.py's reference arm (the FP64 oracle on the host cores) keeps the JSON
contract of the benchmark line; ranks other than 0 exit without work.  CPU only."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(extra_env=None, *args):
    env = dict(os.environ, **(extra_env or {}))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_line_keeps_the_contract():
    r = run(None, "--steps", "1", "--warmup", "1", "--workload", "ant")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["higher_is_better"] is True and d["unit"] == "update steps/s"
    assert d["dtype"] == "f64" and d["vs_baseline"] is None
    assert d["config"]["workload"].startswith("ant_")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_runs_on_rank_zero_only():
    r = run({"RANK": "1", "WORLD_SIZE": "2"}, "--steps", "1", "--warmup", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_oracle_rate_child_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-rate", "0.5", "--workload", "ant"],
                       cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["value"] > 0 and d["steps"] >= 1


def test_default_workload_is_the_large_batch_headline():
    """With no flags the benchmark times the large-batch workload (batch 8192,
    repr 256), reports the roofline of its most expensive kernel class, and adds
    the error against the oracle and the other workloads."""
    sys.path.insert(0, ROOT)
    import bench
    args = bench.build_parser().parse_args([])
    assert args.workload == "large" and bench.WORKLOADS["large"].B == 8192 and bench.WORKLOADS["large"].repr == 256
    assert args.trace == "auto" and not args.no_error and not args.no_extra
    assert args.gpus == 1 and args.warmup >= 3
