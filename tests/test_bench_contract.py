"""The benchmark's output contract, checked on the CPU: the reference arm
(the FP64 oracle on host cores) prints one JSON line with every key the
contract names, and the helpers behind the GPU line's launch count and
kernel names decode the split codes as the library does."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_launch_count_and_kernel_names_follow_the_split_codes():
    # fused: kernel + receivers; marching: two halves + receivers
    assert bench.launches_per_step(2, 106) == 2 and bench.launches_per_step(4, 1432) == 3
    # single-kernel halves, interior / edge halves (2 launches), three-way halves (3)
    assert bench.launches_per_step(1, 2004) == 3
    assert bench.launches_per_step(1, 2285) == 5
    assert bench.launches_per_step(1, 22852324) == 6
    assert bench.launches_per_step(1, 23242324) == 7
    assert bench.split_half_code(22852324, True) == 2285 and bench.split_half_code(22852324, False) == 2324
    assert bench.split_kernel_name(22852324, False) == "str:2324"
    assert bench.kernel_label(1, 22852324) == "split (velocity 2285, stress 2324)"
