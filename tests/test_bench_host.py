"""Host-side parts of bench.py (no GPU): the oracle arm's JSON line keeps the benchmark contract
with the same config dict as our arm, the counted flops follow the block formula of the per-step
work, and the dense oracle's DOF-update rate is measured."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2602_00290_gb300.workloads import plane_config1  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--size", "small",
                          "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "steps/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]
    # the same workload keys as our arm's line (workload_config), so the two lines name one config
    assert d["config"] == json.loads(json.dumps(bench.workload_config(bench.workload("small"))))


def test_counted_flops_block_formula():
    N, r = 1048576, 32
    R1, R2 = 5 * r, r + 1
    assert bench.counted_flops(N, r, r, r) == 2.0 * N * (R1 * R1 + R1 * r + R2 * R2 + R2 * r)


def test_dense_oracle_rate_is_measured():
    wl = plane_config1(nx=8, ny=8, G=4, ntheta=4, nphi=8)
    rate, unknowns, threads, seconds = bench.dense_dof_rate(wl, n=4, reps=2)
    assert unknowns == 4 * 4 * 4 * 4 * 8
    assert rate > 0 and threads >= 1 and seconds > 0


def test_leaf_traffic_is_null_without_a_capture_of_this_source(monkeypatch):
    monkeypatch.setattr(bench, "LEAF_DRAM_96", {("mixed", "column"): (100.0, 50.0, 10)})
    monkeypatch.setattr(bench, "LEAF_DRAM_SOURCE", "0" * 16)  # not the source as it stands
    assert bench.leaf_traffic("mixed", "column", 10, 589824) is None
    monkeypatch.setattr(bench, "LEAF_DRAM_SOURCE", bench.leaf_source_sha())
    assert bench.leaf_traffic("mixed", "column", 10, 589824) == 150.0
    assert bench.leaf_traffic("mixed", "column", 20, 2 * 589824) == 300.0  # rows and leaves scale
    assert bench.leaf_traffic("mixed", "rowsplit", 10, 589824) is None  # no capture of that kernel
