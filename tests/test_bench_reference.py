"""The benchmark's reference arm (the FP64 oracle on the host cores) on CPU: one step over a
one-camera sample (of the relighting workload, to stay quick on CPU) prints a single JSON line with the contract's fields, the same metric and
config as the library arm, and a cpu_baseline that describes the run."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "relight",
                        "--steps", "1", "--warmup", "0", "--ref-cams", "1"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["metric"] == "colorize ms/scene" and d["unit"] == "ms/scene" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "1 of 100 cameras" in d["cpu_baseline"]["sample"]
    # the library arm's config object for the same workload
    assert d["config"]["workload"] == "relight: 200000 Gaussians, 100 cameras 800x800, L=3, 3 channels float32"
    assert d["config"]["parallelism"] == "replicas x1"
