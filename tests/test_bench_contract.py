"""The benchmark's reference arm (the FP64 oracle, OpenMP build, on every host core) prints
one JSON line with the fields of the benchmark contract; runs on CPU in well under a
minute."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, cwd=ROOT,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    sys.path.insert(0, ROOT)
    import bench
    assert line["metric"] == bench.METRIC and line["impl"] == "reference"
    assert line["unit"] == "MLUPS" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["n_gpus"] == 1 and line["steps"] == 1 and line["warmup"] == 0
    assert line["scaling"] == "weak" and line["data"] == "synthetic"
    assert line["config"]["workload"].startswith("couette_suspension_256x256x256")
    assert line["config"]["cells"] == 256 * 256 * 32      # the slab it times
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert cb["cores"] == (os.cpu_count() if "OMP_NUM_THREADS" not in os.environ else cb["cores"])
    assert "slab" in cb["sample"] and "OpenMP" in cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
