"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs, instance by instance (tolerances in tests/parity.py).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_24959_b300 import solver, workloads as W
from tests import parity

pytestmark = pytest.mark.gpu


def _check(w, gpu, idx, what, max_degenerate_frac=0.05):
    ref = oracle.solve_workload(w, idx=idx, threads=8)
    res = parity.compare(w, gpu, ref, idx)
    msg = (f"{what}: worst {res['worst']}, degenerate {res['degenerate']}/"
           f"{res['checked']}, failing {len(res['bad'])} e.g. {res['bad'][:3]}, "
           f"active-set mismatches {res['act_mismatch'][:5]}")
    print(msg)
    assert not res["bad"], msg
    assert res["degenerate"] <= max_degenerate_frac * max(res["checked"], 1), msg
    return res


def test_tiny_full_fused_and_split(cuda_device):
    w = W.tiny()
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    idx = np.arange(w.n)
    _check(w, parity.run_gpu_fused(batch, w), idx, "tiny fused")
    _check(w, parity.run_gpu_split(batch, w), idx, "tiny split")


def test_franka_full(cuda_device):
    w = W.franka()
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    _check(w, parity.run_gpu_fused(batch, w), np.arange(w.n), "franka fused")


def test_quadruped_small_all_instances(cuda_device):
    # several tiles of warps and a ragged tail, every instance checked
    w = W.quadruped(n=1000)
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    _check(w, parity.run_gpu_fused(batch, w), np.arange(w.n), "quadruped-1000 fused")
    _check(w, parity.run_gpu_split(batch, w), np.arange(w.n), "quadruped-1000 split")


def test_quadruped_full_size_sampled(cuda_device):
    """The benchmark's workload (32768 ragged instances) in the benchmark's
    launch configuration (fused, cost-ordered claims); a sample of 2048
    instances is checked against the oracle."""
    w = W.quadruped()
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    order = torch.from_numpy(solver.cost_order(w.inst)).to(cuda_device)
    gpu = parity.run_gpu_fused(batch, w, order=order)
    assert np.all(gpu["status"] == 0), np.bincount(gpu["status"])
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(w.n, 2048, replace=False))
    _check(w, gpu, idx, "quadruped-32768 fused (sampled)")


def test_fused_equals_split_bitwise(cuda_device):
    w = W.quadruped(n=700, seed=77)
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    f = parity.run_gpu_fused(batch, w)
    s1 = parity.run_gpu_split(batch, w, keep_factor=True)
    s0 = parity.run_gpu_split(batch, w, keep_factor=False)
    for k in ("a", "dqfrc", "daref", "dJ", "status", "iters"):
        assert np.array_equal(f[k], s1[k]), k
        assert np.array_equal(s0[k], s1[k]), k


def test_launch_shape_and_order_do_not_change_results(cuda_device):
    w = W.quadruped(n=900, seed=5)
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    base = parity.run_gpu_fused(batch, w)
    order = torch.from_numpy(solver.cost_order(w.inst)).to(cuda_device)
    rev = torch.flip(torch.arange(w.n, dtype=torch.int32, device=cuda_device), [0])
    for kw in (dict(order=order), dict(order=rev), dict(warps_per_block=1),
               dict(warps_per_block=8)):
        o = parity.run_gpu_fused(batch, w, **kw)
        for k in ("a", "dqfrc", "daref", "dJ", "status", "iters"):
            assert np.array_equal(o[k], base[k]), (kw, k)
