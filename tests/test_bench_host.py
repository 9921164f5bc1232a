"""bench.py's host side on the CPU: the command-line defaults the timing
rules ask for (one GPU, at least three warm-up steps), the workload
description, and the reference arm (the FP64 oracle timed on the host
cores) run end to end on a small cloud, printing the JSON line."""
import io
import json
import os
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _args(extra=()):
    old = sys.argv
    sys.argv = ["bench.py", *extra]
    try:
        return bench.parse()
    finally:
        sys.argv = old


def test_defaults_follow_the_timing_rules():
    a = _args()
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1
    assert a.workload == "cloud" and a.impl == "gb300"
    assert (a.n_root, a.levels, a.n_lambda, a.packets_per_bin) == (256, 3, 20, 10_000_000)
    assert bench.NCU_TRACE_BYTES_PER_CROSSING > 0 and bench.NCU_PEEL_BYTES_PER_CROSSING > 0


def test_workload_config_names_the_workload():
    from paper_1206_3710_gb300 import synth
    a = _args(["--n-root", "16", "--levels", "2", "--n-lambda", "3", "--packets-per-bin", "100", "--n-pix", "8"])
    m = bench.make_model(a)
    c = bench.workload_config(a, m)
    assert "molecular cloud: 16^3 root, 2 levels" in c["workload"]
    assert c["n_cells"] == m.tree.n_cells and c["packets_per_step"] == 300
    assert 0 < c["fraction_of_uniform_cells"] <= 1
    assert "L2" in c["l2_policy"]
    assert isinstance(m, synth.Model)


def test_reference_arm_runs_the_oracle(orc):
    a = _args(["--impl", "reference", "--n-root", "16", "--levels", "2", "--n-lambda", "2",
               "--packets-per-bin", "200", "--n-pix", "8", "--cpu-packets-per-bin", "50", "--steps", "2",
               "--warmup", "1"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(a)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT and line["value"] > 0
    assert line["steps"] == 2 and line["warmup"] == 1 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("molecular cloud: 16^3 root")
