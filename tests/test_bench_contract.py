"""The benchmark's JSON line: the reference arm (the FP64 oracle on the host
cores, runs without a GPU) and, on a GPU, our arm's required keys; and the
algorithmic work formulas the roofline divides by."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2607_24959_b300 import workloads as W  # noqa: E402


def _line(args, timeout):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT,
                       capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _line(["--impl", "reference", "--steps", "1", "--warmup", "0"], 600)
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["config"]["instances"] == 32768


def test_work_formulas():
    w = W.quadruped(n=256, seed=5)
    k = np.full(w.n, 7)
    act = (w.inst["m"] // 2).astype(np.int64)
    f, b = bench.algorithmic_work(w.inst, k, act)
    f2, _ = bench.algorithmic_work(w.inst, 2 * k, act)
    assert f > 0 and b > 0 and f2 > f                   # work grows with the steps
    nv, m = w.inst["nv"].astype(float), w.inst["m"].astype(float)
    # bytes: M lower, J, the vectors and the outputs, each once, 4 B each
    exp = 4 * (nv * (nv + 1) / 2 + 2 * m * nv + 4 * nv + 3 * m)
    assert abs(b - exp.sum()) <= 1e-9 * b
    we = W.quadruped_elliptic(n=256, seed=6)
    fe, be = bench.elliptic_work(we.inst, np.full(we.n, 12), we.inst["m"] // 3)
    assert fe > 0 and be > 0
    fn, bn = bench.ncg_work(w.inst, np.full(w.n, 900), act)
    assert fn > 20 * f and bn == b                      # hundreds of cheaper CG steps, same bytes


@pytest.mark.gpu
def test_our_arm_line(cuda_device):
    d = _line(["--steps", "5", "--warmup", "3", "--warmup-seconds", "0", "--no-serve",
               "--no-memory", "--no-elliptic", "--no-ncg", "--configs", "tiny",
               "--cpu-sample", "2048", "--e2e-chunks", "2"], 900)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches", "configs"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 5 and d["scaling"] == "weak"
    r = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert 0 < r["frac"] < 1 and abs(r["achieved"] / r["peak"] - r["frac"]) < 1e-9
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] >= d["steps"]
    assert "roofline" in d["configs"]["tiny"] and d["configs"]["tiny"]["value"] > 0
    for k in ("sm_mhz", "sm_max_mhz", "reasons"):
        assert k in d["clocks"], k


@pytest.mark.gpu
def test_serve_leg_line(cuda_device):
    """The serving leg on a short stream: both policies complete every
    request (the leg raises if one is lost; a rare hard instance may stop at
    the iteration cap instead of converging), and each reports its latency
    split (client lag, queue, service) and its p50 / p99 per nv class."""
    d = _line(["--steps", "3", "--warmup", "3", "--warmup-seconds", "0", "--no-e2e",
               "--no-cpu-baseline", "--no-memory", "--no-elliptic", "--no-ncg", "--configs", "",
               "--serve-requests", "20000", "--serve-sweep", ""], 900)
    s = d["serve"]
    assert s["requests"] == 20000
    for pol in ("continuous", "fixed_1024"):
        r = s[pol]
        assert r["ok"] >= 0.999 * 20000 and r["solves_per_s"] > 0, (pol, r["ok"])
        assert 0 < r["p50_ms"] <= r["p99_ms"], pol
        split = r["latency_split"]
        for k in ("client_lag", "queue", "service"):
            assert split[k]["p50_ms"] <= split[k]["p99_ms"], (pol, k)
        assert set(split["by_nv"]) == {3, 9, 18, 96} or set(split["by_nv"]) == {"3", "9", "18", "96"}
