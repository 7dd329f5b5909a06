"""bench.py's JSON contract on CPU: the reference arm (the oracle on the host) prints one line with the
required keys; workload configs and the kernel-source digest are well formed; the op-count model is
consistent between the two methods."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2311_14941_gb300 import chem, opcount, synth  # noqa: E402


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["metric"] == bench.METRIC
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_workload_configs_and_digest():
    for name in bench.WORKLOADS:
        c = bench.config(name, "persistent")
        assert c["n_cells"] > 0 and c["rtol"] == bench.RTOL and "workload" in c and "state" in c
    d = bench.kernel_sources_digest()
    assert len(d) == 16 and int(d, 16) >= 0


def test_opcount_methods():
    m = synth.mechanism_methane_sized()
    h = chem.create(m, device=-1)
    a = opcount.model(m, h.export_plan(0), h.export_plan(1), method=0)
    b = opcount.model(m, h.export_plan(0), h.export_plan(1), method=1)
    assert a.f_eval == b.f_eval and a.jac == b.jac and a.lu == b.lu
    # RODAS3 has one more right-hand side and two more stage solves per attempt than ROS2
    assert a.attempt - b.attempt >= a.f_eval + 2 * a.solve
    c = opcount.model(m, h.export_plan(0), h.export_plan(1), method=2)
    # RODAS4: three more right-hand sides and two more stage solves per attempt than RODAS3
    assert c.f_eval == a.f_eval and c.jac == a.jac
    assert c.attempt - a.attempt >= 3 * a.f_eval + 2 * a.solve
    s = a.cell_slots(np.array([10, 20]), np.array([9, 18]))
    assert np.allclose(s, [10 * a.attempt + 9 * a.jac, 20 * a.attempt + 18 * a.jac])
    assert abs(opcount.fp64_peak_tflops() - 2 * 152 * 2.07 * 2 / 1e3) < 1e-12


def test_cpu_baseline_reports_all_cores_and_one_core():
    m = synth.mechanism_small()
    F = synth.field_uniform_random(m, 64, seed=3)
    b = bench.cpu_baseline(m, F, "small test", budget_s=0.2)
    assert b["kind"] == "oracle" and b["unit"] == "reactor-steps/s" and b["value"] > 0 and b["cores"] >= 1
    one = b["single_core"]
    assert one["cores"] == 1 and one["value"] > 0 and "cells" in one["sample"]
