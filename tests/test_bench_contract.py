"""The parts of bench.py's output that need no GPU: the reference arm's JSON line (the
oracle on the host's cores) and the lookup of committed DRAM traffic records."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "0", "--n", "4096"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    # ms_per_step is the time of the bounded steps this run timed
    assert line["ms_per_step"] * line["steps"] == pytest.approx(1e3 * line["wall_s"], rel=1e-9)
    assert line["full_step_ms_extrapolated"] == pytest.approx(1e3 * 4096 / line["value"])


def test_traffic_records_match_kernel_and_schedule(tmp_path, monkeypatch):
    import bench

    recs = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    src = os.path.join(ROOT, "paper_1212_2934_gb300", "csrc", "k_field.cu")
    for d in recs:
        got = bench.traffic_for(src, d["n"], d["workload_name"], d["theta"], d["leaf_max"],
                                d["schedule"], kernel=d.get("kernel", "k_bh"))
        assert got == d["dram_bytes_per_launch"]
    # another schedule, workload or kernel has no record
    d = recs[0]
    assert bench.traffic_for(src, d["n"], d["workload_name"], d["theta"], d["leaf_max"], 99,
                             kernel=d.get("kernel", "k_bh")) is None
    assert bench.traffic_for(src, d["n"], "chains", d["theta"], d["leaf_max"], d["schedule"],
                             kernel=d.get("kernel", "k_bh")) is None
    # a changed source has no record
    changed = tmp_path / "k_field.cu"
    changed.write_bytes(open(src, "rb").read() + b"\n")
    assert bench.traffic_for(str(changed), d["n"], d["workload_name"], d["theta"],
                             d["leaf_max"], d["schedule"], kernel=d.get("kernel", "k_bh")) is None
