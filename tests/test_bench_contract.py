"""The bench's JSON line: the keys and types every run must print.

The reference arm (the oracle on the host cores, a bounded sample) runs on the
CPU; the default arm runs on a GPU (a short run of the same workload)."""
import json
import math
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASE = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config")


def _run(*args, timeout=900):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                       text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def _check_base(d, steps, warmup):
    for k in BASE:
        assert k in d, k
    assert d["value"] > 0 and math.isfinite(d["value"])
    assert d["unit"] == "path-steps/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == steps and d["warmup"] == warmup
    assert d["scaling"] == "weak" and d["data"] == "synthetic"
    assert isinstance(d["config"], dict) and d["config"].get("workload")


def test_reference_arm_line():
    d = _run("--impl", "reference", "--steps", "1", "--warmup", "0", timeout=300)
    _check_base(d, 1, 0)
    assert d["impl"] == "reference" and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.mark.gpu
def test_default_arm_line():
    d = _run("--steps", "4", "--warmup", "3", "--no-cpu", "--no-cv")
    _check_base(d, 4, 3)
    assert d["dtype"] == "f32" and d["vs_baseline"] is None
    r = d["roofline"]
    assert r["bound"] == "alu" and r["unit"] == "Tops/s"
    assert 0 < r["frac"] < 1.2 and r["achieved"] > 0 and r["peak"] > 0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    e = d["e2e"]
    assert e["value"] > 0 and e["unit"] == d["unit"] and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] > 0
    assert "clocks" in d


def test_profiled_counters_follow_the_sources(tmp_path):
    # the roofline's traffic and issue-slot figures come from a committed ncu summary only while
    # the kernel's sources hash to what the summary records
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "kernel.cu"
    src.write_text("// a kernel\n")
    rel = os.path.relpath(str(src), ROOT)
    h = hashlib.sha256(src.read_bytes()).hexdigest()
    prof = tmp_path / "k.md"
    prof.write_text("| issue-slot utilisation (`smsp__issue_active.avg.pct_of_peak_sustained_active`) | 70.5 % |\n"
                    f"dram_bytes_per_launch: 1234\npath_steps_per_launch: 10\nsource_sha256: {h}\nsources: {rel}\n")
    got = bench.profiled_counters(str(prof))
    assert got == {"dram_bytes_per_launch": 1234.0, "path_steps_per_launch": 10.0, "issue_slots": 0.705}
    src.write_text("// the kernel changed\n")
    assert bench.profiled_counters(str(prof)) is None
    assert bench.profiled_counters(str(tmp_path / "absent.md")) is None
