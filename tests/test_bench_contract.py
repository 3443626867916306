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
    """bench.traffic_for returns a record's DRAM bytes only for the same kernel, source
    (by hash), workload and launch schedule."""
    import hashlib

    import bench

    src = tmp_path / "k_field.cu"
    src.write_bytes(b"// a kernel source\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    recs = [dict(kernel="k_bh", source_sha256=sha, n=1024, workload_name="phi05", theta=0.5,
                 leaf_max=1, schedule=2, dram_bytes_per_launch=111),
            dict(kernel="k_bh_rec", source_sha256=sha, n=1024, workload_name="grad", theta=0.5,
                 leaf_max=1, schedule=0, dram_bytes_per_launch=222)]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(recs))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for(str(src), 1024, "phi05", 0.5, 1, 2) == 111
    assert bench.traffic_for(str(src), 1024, "grad", 0.5, 1, 0, kernel="k_bh_rec") == 222
    assert bench.traffic_for(str(src), 1024, "phi05", 0.5, 1, 1) is None        # schedule
    assert bench.traffic_for(str(src), 1024, "chains", 0.5, 1, 2) is None       # workload
    assert bench.traffic_for(str(src), 2048, "phi05", 0.5, 1, 2) is None        # size
    assert bench.traffic_for(str(src), 1024, "grad", 0.5, 1, 0) is None         # kernel
    src.write_bytes(b"// the kernel source, changed\n")
    assert bench.traffic_for(str(src), 1024, "phi05", 0.5, 1, 2) is None        # source
