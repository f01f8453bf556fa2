"""The benchmark's JSON line: the reference arm (the oracle on the host cores, no GPU) and the
GPU arm carry every key of the reporting contract with consistent values."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COMMON = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
          "vs_baseline", "dtype", "data", "config")


def run_bench(*args, timeout=600):
    r = subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, capture_output=True, text=True,
                       timeout=timeout)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = run_bench("--impl", "reference", "--steps", "1", "--warmup", "3")
    for k in COMMON + ("impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 3
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


@pytest.mark.gpu
def test_gpu_arm_line():
    steps = 6
    d = run_bench("--steps", str(steps), "--warmup", "3", "--no-cpu", "--no-extra", "--no-autotune")
    for k in COMMON + ("roofline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["scaling"] == "weak" and d["dtype"] == "f32" and d["value"] > 0
    # value = cells x 3 stages x steps / device time
    cells = d["config"]["cells_per_gpu"]
    assert d["value"] == pytest.approx(cells * 3 * steps / (d["ms_per_step"] * steps * 1e-3) / 1e9, rel=1e-9)
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] > 0
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-12)
    # achieved = algorithmic bytes of one launch / its measured duration
    assert r["achieved"] == pytest.approx(r["bytes_per_cell_stage"] * cells / (r["launch_ms"] * 1e-3) / 1e9,
                                          rel=1e-9)
    assert r["traffic"] is None or r["traffic"] > 0
    assert d["gpu_launches"] == 3 * steps
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] == e["d2h_bytes_per_step"] == 4 * 4 * cells
    assert e["float64_host_arrays"]["h2d_bytes_per_step"] == 8 * 4 * cells
    c = d["clocks"]
    assert "sm_mhz" in c and "sm_max_mhz" in c and isinstance(c["reasons"], list)


def test_gpus_flag_and_world_size_must_agree():
    """--gpus N and a launcher's WORLD_SIZE must agree, and without a launcher bench.py starts N
    ranks itself only when N GPUs are visible; a mismatch exits non-zero before any work."""
    env = dict(os.environ, WORLD_SIZE="2", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, "bench.py", "--gpus", "1", "--steps", "1"], cwd=ROOT, capture_output=True,
                       text=True, env=env, timeout=300)
    assert r.returncode != 0 and "WORLD_SIZE" in r.stderr
    import torch
    if torch.cuda.device_count() < 64:
        env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
        r = subprocess.run([sys.executable, "bench.py", "--gpus", "64", "--steps", "1"], cwd=ROOT,
                           capture_output=True, text=True, env=env, timeout=300)
        assert r.returncode != 0 and "visible" in r.stderr


@pytest.mark.gpu
def test_warped_slabs_line():
    """The strong-scaling slab workload on one GPU (one slab, the same stage-part path)."""
    d = run_bench("--workload", "warped-slabs", "--steps", "4", "--warmup", "3")
    for k in COMMON + ("roofline", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["scaling"] == "strong" and d["n_gpus"] == 1 and d["value"] > 0
    assert d["config"]["cells"] == 4096 * 4096
