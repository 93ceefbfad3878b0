"""bench.py's reference arm (the FP64 oracle on the host cores) prints one JSON line with the
fields of the benchmark contract, with the metric and config keys of the GPU arm, for both
workloads.  Its value is the time it measured on the bounded sample that it names in
config.workload (the full workload it samples is named beside it); a DOF-ratio extrapolation
appears only in its own labelled field.  CPU only (one step, no warm-up)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("cfg,n_full,nrhs,tag", [(2, 2_099_200, 1, "256x256"), (4, 2_738_019, 16, "48^3")])
def test_reference_arm_json_line(cfg, n_full, nrhs, tag):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--cfg", str(cfg)], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "s"
    assert d["higher_is_better"] is False and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    c = d["config"]
    sample = bench.workload(bench.WORKLOADS[cfg]["sample_N"], cfg)
    assert c["n_dofs"] == sample["n"] and c["workload"] == bench.workload_name(sample)
    assert c["sample_of_dofs"] == n_full and tag in c["sample_of"] and c["nrhs"] == nrhs
    assert d["dof_scaled_lower_bound_s"] == pytest.approx(d["value"] * n_full / sample["n"])
    assert {"workload", "n_dofs", "nrhs", "solve_mode", "options", "l2", "parallelism"} <= set(c)


def test_l2_note_flags_reduced_sizes():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.l2_note(bench.workload(256)).startswith("inputs larger than L2")
    assert bench.l2_note(bench.workload(16)).startswith("inputs smaller than L2")


def test_throughput_entry():
    sys.path.insert(0, ROOT)
    import bench
    t = bench.throughput_entry(2_000_000, 16, 10.0, 4.0, [10, 12])
    assert t["setup_dofs_per_s"] == 200_000.0
    assert t["solve_dof_iterations_per_s"] == 2_000_000 * 16 * 11.0 / 4.0
    assert t["iterations"] == 11.0
    z = bench.throughput_entry(5, 1, 0.0, 0.0, [])
    assert z["setup_dofs_per_s"] is None and z["solve_dof_iterations_per_s"] is None
    json.dumps(t)
