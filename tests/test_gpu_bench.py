"""bench.py end to end on the GPU at a small size: the JSON line the round-end
run parses, with every object the contract asks for, and more bench steps
than one system may run (the schedule starts fresh systems), so that a
change that breaks the bench shows here first."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu


def test_bench_line_small():
    from paper_2201_01446_gb300 import dp  # noqa: F401  (builds the library first)
    cmd = [sys.executable, "bench.py", "--cells", "10", "--steps", "12", "--warmup", "3",
           "--plain-steps", "2", "--e2e-steps", "1", "--serve-requests", "10",
           "--serve-capacity-requests", "5", "--grad-cells", "6", "--water-reps", "2",
           "--water-steps", "1"]
    env = dict(os.environ, DP_SKIP_BUILD="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "dtype", "data", "config", "gpu_launches",
                "roofline", "cpu_baseline", "e2e", "clocks", "fp32_peak", "plain", "serve"):
        assert key in d, key
    assert d["steps"] == 12 and d["warmup"] == 3 and d["value"] > 0
    assert d["config"]["systems"] == 2  # 12 blocks: two fresh systems
    assert d["gpu_launches"] > 0
    rf = d["roofline"]
    assert rf["bound"] == "alu" and 0 < rf["frac"] and rf["peak"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert d["accuracy_vs_oracle"]["within_bars"]
    assert d["serve"]["errors"] == 0 and d["serve"]["requests"] == 10
    assert d["plain"]["roofline"]["embed_contract_fwd"]["frac"] > 0
