"""The reference arm of the benchmark (`bench.py --impl reference`) times the FP64 oracle on the
host, on the same workload as the GPU arm: it must print one JSON line carrying the keys the
GPU arm carries, with the oracle described as the CPU baseline and no host-device copies.
One timed iteration of the full 384 x 256 grid on one core (a few seconds)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_complete_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["metric"] == "Mcell-iter/s" and d["unit"] == "Mcell-iter/s" and d["higher_is_better"]
    assert d["steps"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    # the same workload as the GPU arm's line
    assert d["config"]["workload"].startswith("half-cylinder-384x256-air11")
    assert d["config"]["cells"] == 384 * 256
