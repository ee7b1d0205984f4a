"""The benchmark's output line: one JSON object with the keys its consumers read.
The reference arm (the oracle on the host cores) runs on CPU; the GPU arm needs a
device."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, timeout=600):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=timeout)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


COMMON = ["metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
          "scaling", "vs_baseline", "dtype", "data", "config", "e2e"]


def test_reference_arm_line():
    d = run_bench("--impl", "reference", "--steps", "1", "--warmup", "1")
    for k in COMMON + ["impl", "cpu_baseline"]:
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert "workload" in d["config"]
    # the reference arm times the GPU arm's own workload (default precision: fp32x2)
    sys.path.insert(0, ROOT)
    import bench
    assert d["config"] == dict(bench.config("fp32x2"), parallelism="single")


@pytest.mark.gpu
def test_gpu_arm_line():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():  # pragma: no cover
        pytest.skip("needs a CUDA device")
    d = run_bench("--steps", "5", "--warmup", "3", "--no-cpu-baseline", "--no-t-final", "--no-fft")
    for k in COMMON + ["roofline", "clocks", "gpu_launches", "kernels"]:
        assert k in d, k
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 5
    r = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert r["bound"] in ("hbm", "tensor", "alu") and 0 < r["frac"] < 2
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] >= 5 * d["steps"]
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])


def test_sweep_interpolation_helpers():
    # the error-against-cost summary interpolates a power law exactly in log-log
    sys.path.insert(0, ROOT)
    import bench

    xs = [1e-1, 1e-2, 1e-3]
    ys = [x ** -0.5 for x in xs]
    assert abs(bench._loglog_at(xs, ys, 3e-2) - 3e-2 ** -0.5) < 1e-12
    assert abs(bench._loglog_at(xs[::-1], ys[::-1], 5e-3) - 5e-3 ** -0.5) < 1e-12
    assert bench._loglog_at(xs, ys, 1.0) is None
    assert abs(bench._slope(xs, ys) + 0.5) < 1e-12
    assert bench._slope([1.0], [2.0]) is None


def test_morphology_counts_on_the_periodic_grid():
    # loops (one hole each), a disc, and a loop that wraps around the corner
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench

    n = 128
    y, x = np.mgrid[0:n, 0:n]

    def ring(cx, cy, r0, r1):
        dx = np.minimum(abs(x - cx), n - abs(x - cx))
        dy = np.minimum(abs(y - cy), n - abs(y - cy))
        r = np.hypot(dx, dy)
        return (r > r0) & (r < r1)

    u = -np.ones((n, n))
    u[ring(64, 64, 20, 26)] = 0.5
    assert bench._topology(u) == (1, 1)
    u[ring(2, 2, 8, 12)] = 0.5
    assert bench._topology(u) == (2, 2)
    u[ring(100, 30, -1, 4)] = 0.5
    assert bench._topology(u) == (3, 2)
    band = -np.ones((n, n))
    band[:, 60:64] = 0.5
    assert bench._topology(band) == (1, 0)
