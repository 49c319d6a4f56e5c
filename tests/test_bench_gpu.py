"""bench.py's JSON line on the GPU: the keys and their relations that the
measurement contract fixes (one line, rank 0, K timed steps, roofline against
the measured copy bandwidth, clocks sampled during the timed region)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


@pytest.mark.parametrize("storage,launches", [("f32", 1), ("f16s", 2)])
def test_bench_line_keeps_the_contract(storage, launches):
    d = _run("--steps", "10", "--warmup", "3", "--no-extras", "--storage", storage)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["unit"] == "MFLUPS" and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["steps"] == 10 and d["warmup"] == 3 and d["gpu_launches"] == 10 * launches
    assert d["dtype"] == "f32" and d["data"] == "synthetic" and "workload" in d["config"]
    n_fluid = d["config"]["n_fluid"]
    assert abs(d["value"] - n_fluid / (d["ms_per_step"] * 1e-3) / 1e6) <= 1e-6 * d["value"]
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] > 0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) <= 1e-12
    assert abs(r["achieved"] - r["alg_bytes_per_launch"] / (d["ms_per_step"] * 1e-3) / 1e9) <= 1e-6 * r["achieved"]
    c = d["clocks"]
    assert c["samples"] >= 1 and c["sm_mhz"] is not None
    assert d["status_word"] == 0
    t = d["timing"]
    assert t["sub_regions"] == 5 and t["min_ms"] <= t["median_ms"] <= t["max_ms"]
