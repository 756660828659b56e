"""GPU parity of the one-CTA-per-instance kernels (nv > 32 or m > 256):
the scaling-extreme workloads (nv = 96 with cond(M) = 1e4; m = 1024 rows) and
ragged batches that mix warp- and CTA-sized instances."""
import numpy as np
import pytest
import torch

from paper_2607_24959_b300 import solver, workloads as W
from tests import parity
from tests.test_gpu_parity import _check

pytestmark = pytest.mark.gpu


def test_nv96_sampled(cuda_device):
    w = W.nv96()                                  # 2048 x nv 96, m 64, cond 1e4
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    gpu = parity.run_gpu_fused(batch, w)
    assert np.all(gpu["status"][:w.n] == 0), np.bincount(gpu["status"][:w.n])
    idx = np.sort(np.random.default_rng(1).choice(w.n, 256, replace=False))
    _check(w, gpu, idx, "nv96 fused (sampled)")


def test_nc256_all(cuda_device):
    w = W.nc256()                                 # 256 x nv 18, m 1024
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    gpu = parity.run_gpu_fused(batch, w)
    _check(w, gpu, np.arange(w.n), "nc256 fused")


def test_cta_split_equals_fused_bitwise(cuda_device):
    w = W.generate("cta", 120, 40, 75, seed=41, cond=1e3)   # nv 40, m 300 (2 rows/thread)
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    f = parity.run_gpu_fused(batch, w)
    s1 = parity.run_gpu_split(batch, w, keep_factor=True)
    s0 = parity.run_gpu_split(batch, w, keep_factor=False)
    _check(w, f, np.arange(w.n), "cta nv40 m300")
    masks = parity.valid_mask(w)
    # the CTA solver rebuilds the Newton matrix in full in every mode, so the
    # three paths share the forward and the adjoint solve bit for bit; f in
    # dJ differs in its last bits where a fused solve stopped after a
    # refinement step (f advanced along it; the split adjoint re-evaluates it)
    for k in ("a", "dqfrc", "daref", "status", "iters"):
        assert np.array_equal(parity.valid(w, f, k, masks), parity.valid(w, s1, k, masks)), k
        assert np.array_equal(parity.valid(w, s0, k, masks), parity.valid(w, s1, k, masks)), k
    assert np.array_equal(parity.valid(w, s0, "dJ", masks), parity.valid(w, s1, "dJ", masks))
    x = parity.valid(w, f, "dJ", masks).astype(np.float64)
    y = parity.valid(w, s1, "dJ", masks).astype(np.float64)
    assert np.max(np.abs(x - y)) <= 1e-6 * max(np.max(np.abs(y)), 1e-30)


def test_plan_mixes_warp_and_cta_buckets(cuda_device):
    parts = []
    for gen in (lambda: W.quadruped(n=300, seed=51),
                lambda: W.generate("big", 40, 96, 20, seed=52, cond=1e4),
                lambda: W.generate("rows", 30, 18, 100, seed=53, cond=1e3),
                lambda: W.generate("mid", 40, 33, 10, seed=54, cond=1e3)):
        w = gen()
        parts += [w.instance(b) for b in range(w.n)]
    rng = np.random.default_rng(2)
    w = W.pack([parts[i] for i in rng.permutation(len(parts))], name="warp+cta")
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    g = torch.from_numpy(w.g).to(cuda_device)
    plan = solver.FusedPlan(batch, g, autotune=True, graph=True)
    kinds = {b["kernel"] for b in plan.describe()["buckets"]}
    assert kinds == {"warp", "cta"}, plan.describe()
    out = plan.launch()
    torch.cuda.synchronize()
    gpu = dict(a=out.a.cpu().numpy(), dqfrc=out.dqfrc.cpu().numpy(),
               daref=out.daref.cpu().numpy(), dJ=out.dJ.cpu().numpy(),
               status=out.status.cpu().numpy(), iters=out.iters.cpu().numpy())
    _check(w, gpu, np.arange(w.n), "warp + cta plan")
    plan.close()
