"""The benchmark's reference arm (the CPU oracle on the host cores) runs
without a GPU and prints the contract's JSON line."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
         "--warmup", "3", "--nx", "64", "--ny", "16"],
        capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "cell-updates/s" and d["value"] > 0
    assert d["metric"] == "2D Euler GP-MOOD cell-updates/s" and d["higher_is_better"] is True
    assert d["warmup"] <= 3 and d["steps"] >= 1 and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == os.cpu_count()
    assert cb["value"] == d["value"] and cb["single_thread"]["cores"] == 1
    assert cb["single_thread"]["value"] > 0 and cb["host"]["nproc"] == os.cpu_count()
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    # the workload is the full double Mach reflection; each step of the
    # oracle is a step of the same problem on the sample grid
    assert d["config"]["cells"] == 4096 * 1024 and d["cpu_baseline"]["sample_cells"] == 64 * 16
    assert d["config"]["parallelism"] == "replicas x1"
