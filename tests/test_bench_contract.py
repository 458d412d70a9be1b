"""bench.py prints one JSON line with the keys its consumers read: the reference arm
(FP64 oracle on the host cores) on the CPU, the GPU arm on a small batch on a GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASE_KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
             "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e")


def _run(args, timeout):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                       capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run(["--impl", "reference", "--instances", "8", "--steps", "1", "--warmup", "1"], 600)
    for k in BASE_KEYS + ("impl", "cpu_baseline"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert "workload" in d["config"]
    for k in ("value", "cores", "kind", "sample"):
        assert k in d["cpu_baseline"], k
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


@pytest.mark.gpu
def test_gpu_arm_line():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = _run(["--instances", "64", "--steps", "2", "--warmup", "3", "--serve-requests", "4",
              "--no-others", "--cpu-sample", "8", "--lanes", "2"], 1800)
    for k in BASE_KEYS + ("roofline", "cpu_baseline", "gpu_launches", "clocks", "fp64",
                          "fp32_bulk_accuracy", "serving"):
        assert k in d, k
    assert d["value"] > 0 and d["steps"] == 2 and d["n_gpus"] == 1 and d["gpu_launches"] > 0
    r = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in d["e2e"], k
    assert d["e2e"]["h2d_bytes_per_step"] == 12 * 8 * d["config"]["cells"]
    for k in ("sm_mhz", "sm_max_mhz", "reasons"):
        assert k in d["clocks"], k
    assert d["serving"]["completed"] == 4
