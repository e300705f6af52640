"""Host-side contract of bench.py (no GPU): the byte accounting behind the
roofline fields, the source-keyed DRAM traffic figure, and the reference arm's
JSON line (the FP64 oracle on the host cores)."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_method_and_design_bytes():
    # read + write of 38 populations at the storage width
    assert bench.method_bytes_per_lu("fp64") == 608
    assert bench.method_bytes_per_lu("fp32") == 304
    assert bench.method_bytes_per_lu("fp16") == bench.method_bytes_per_lu("bf16") == 152
    # collision: 19 pulled + 19 written populations, phi, n, |grad phi|, kappa in, the 4-real record out
    assert bench.design_bytes_per_node("collide", "fp32") == 38 * 4 + 10 * 4 == 192
    assert bench.design_bytes_per_node("collide", "fp16") == 38 * 2 + 10 * 4 == 116
    # order parameter: 19 pulled populations, the sources' records (4 reals) and phi out
    assert bench.design_bytes_per_node("phi", "fp32") == 19 * 4 + 5 * 4 == 96
    assert bench.design_bytes_per_node("grad_wetting", "fp32") == 24
    assert bench.population_bytes_per_node("collide", "fp32") == 152


def test_traffic_figure_is_keyed_to_the_fluid_sources(monkeypatch):
    h = bench.fluid_source_hash()
    assert len(h) == 16 and h == bench.fluid_source_hash()
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {("collide", "fp32"): (123, h)})
    assert bench.ncu_traffic("collide", "fp32") == 123
    assert bench.ncu_traffic("collide", "fp16") is None
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {("collide", "fp32"): (123, "0" * 16)})
    assert bench.ncu_traffic("collide", "fp32") is None


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3  # at least 3 warm-up steps, whatever is asked
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["metric"] == bench.METRIC and d["config"]["workload"] == bench.WORKLOAD
