"""bench.py's output contract: one JSON line with the keys the measurement needs.  The
reference arm (the oracle on the host cores) runs here on the CPU; the GPU arm on a small
configuration under the gpu marker."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
             "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline"}


def run_bench(*args, timeout=900):
    out = subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, capture_output=True, text=True,
                         timeout=timeout)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    d = run_bench("--impl", "reference", "--steps", "1", "--warmup", "1", "--ref-sample", "10")
    assert BASE_KEYS <= set(d) and d["impl"] == "reference"
    assert d["warmup"] >= 3 and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


@pytest.mark.gpu
def test_gpu_arm_line():
    d = run_bench("--steps", "3", "--warmup", "3", "--N", "16", "--no-autotune", "--sampler-traj", "0",
                  "--batched-req", "0", "--served=", "--walltime-m=", "--dense-samples", "0",
                  "--cpu-sample", "12")
    assert BASE_KEYS <= set(d) and {"roofline", "gpu_launches", "clocks"} <= set(d)
    r = d["roofline"]
    assert r["bound"] == "alu" and 0 < r["frac"] < 1.5 and r["achieved"] > 0 and r["peak"] > 0
    assert d["gpu_launches"] > 0 and d["value"] > 0 and d["e2e"]["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"


def test_fx_product_model():
    # the closed sum over depths equals the recursion over the tree's nodes, and the one- and
    # two-mode trees come out at their hand counts
    sys.path.insert(0, ROOT)
    import bench
    R, SG = 89.0 / 26.0, 39.0 / 26.0

    def walk(m):  # products below (and including) one node with m undecided modes
        if m == 1:
            return 2.0 + R + SG
        t = m - 1
        here = 2.0 + R + 1.0 + 3.0 + SG + 8.0 * t + 2.0 * t * (2 * t + 1)
        return here + 2.0 * walk(m - 1)

    assert bench.fx_products(1) == 2.0 + R + SG
    assert bench.fx_products(2) == (2.0 + R + 1.0 + 3.0 + SG + 8.0 + 6.0) + 2.0 * (2.0 + R + SG)
    for n in range(1, 16):
        assert abs(bench.fx_products(n) - walk(n)) <= 1e-9 * walk(n)
