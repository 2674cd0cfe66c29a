"""The bench line on a GPU: one JSON line with the contract's keys and a
roofline object whose fraction is achieved / peak (profiler counters only
when they were taken on the kernel sources being run)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_quick_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--quick", "--steps", "3",
                          "--warmup", "3", "--n", "200000"], capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "gpu_launches", "clocks", "roofline"):
        assert key in d, key
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3
    assert d["value"] > 0 and d["gpu_launches"] > 0 and d["dtype"] == "f64"
    r = d["roofline"]
    assert r["bound"] == "alu" and r["peak"] > 0            # measured in the run
    if r["ncu_sources"] == r["kernel_sources"]:
        assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    else:   # counters of another kernel build are not reported
        assert r["achieved"] is None and r["frac"] is None and r["traffic"] is None
    h = d["hbm_roofline"]
    assert h["frac"] == pytest.approx(h["achieved"] / h["peak"])
    c = d["clocks"]
    assert c["sm_max_mhz"] > 0 and isinstance(c["reasons"], list)
