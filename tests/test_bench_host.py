"""Host logic of bench.py, without a GPU.

* the reference arm (the oracle on all host cores: one spawned process per core,
  a disjoint share of one block sample each, passes started from a common
  barrier) prints the contract's line with the GPU arm's config, and its value
  is the sample's bytes over the median pass;
* the serving draw is seeded, stays inside its ranges and alternates the two
  kernels;
* the CPU model is read from the host.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "3", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, PYTHONPATH=ROOT))
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "GB/s"
    assert line["steps"] == 3 and line["warmup"] == 3 and line["higher_is_better"] is True
    assert line["config"] == bench.config_of(bench.N_DEFAULT, 1)
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == (os.cpu_count() or 1) and cb["nproc"] == cb["cores"]
    assert cb["value"] == line["value"] > 0
    assert line["e2e"] == {"value": line["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert abs(line["ms_per_step"] * 1e-3 * line["value"] * 1e9 - float(cb["sample"].split("MB algorithmic")[0]
                                                                            .split(",")[-1].split()[-1]) * 1e6) \
        <= 0.02 * line["value"] * line["ms_per_step"] * 1e6


def test_cpu_baseline_splits_one_sample():
    """Two processes time disjoint halves of the same sample: their bytes add up to the
    one-process sample's bytes."""
    one = bench.cpu_baseline_parallel(0.4, 2, 0, workers=1, n=16384)
    two = bench.cpu_baseline_parallel(0.2, 2, 0, workers=2, n=16384)
    assert one["alg_bytes"] == two["alg_bytes"] > 0
    assert one["cores"] == 1 and two["cores"] == 2


@pytest.mark.parametrize("lo,hi", [(16384, 131072), (16384, 1048576)])
def test_serving_draw(lo, hi):
    d = bench.serving_draw(lo, hi)
    assert d == bench.serving_draw(lo, hi)                      # seeded
    assert len(d) == 8
    assert [k for k, _, _ in d] == ["laplace", "matern"] * 4
    for _, n, eps in d:
        assert n % 1024 == 0 and lo - 1024 <= n <= hi + 1024
        assert eps in (1e-4, 1e-6, 1e-8)


def test_cpu_model_named():
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()
