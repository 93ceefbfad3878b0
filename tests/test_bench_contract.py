"""bench.py's reference arm (the FP64 oracle on the host cores) prints one JSON line with the
fields of the benchmark contract, on the same workload, metric and config keys as the GPU
arm.  CPU only (a one-step, no-warm-up run on the bounded 16x16 sample)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
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
    cfg = d["config"]
    assert cfg["n_dofs"] == 2_099_200 and "256x256" in cfg["workload"]
    assert cfg["l2"].startswith("inputs larger than L2")
    assert {"workload", "n_dofs", "solve_mode", "options", "l2", "parallelism"} <= set(cfg)


def test_l2_note_flags_reduced_sizes():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.l2_note(bench.workload(256)).startswith("inputs larger than L2")
    assert bench.l2_note(bench.workload(16)).startswith("inputs smaller than L2")
