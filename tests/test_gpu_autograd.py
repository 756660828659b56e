"""torch.autograd.Function wrapper: its backward is the IFT adjoint kernel,
checked against the FP64 oracle; adjoint-state memory is flat in the Newton
iteration cap K (Section III-D: no solver trace is stored)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_24959_b300 import autograd as csag, solver, workloads as W
from tests import parity

pytestmark = pytest.mark.gpu


def test_autograd_matches_oracle(cuda_device):
    w = W.franka(n=512, seed=21)
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    J = batch.J.clone().requires_grad_(True)
    q = batch.qfrc.clone().requires_grad_(True)
    ar = batch.aref.clone().requires_grad_(True)
    a = csag.contact_solve(batch, J=J, qfrc=q, aref=ar)
    g = torch.from_numpy(w.g).to(cuda_device)
    loss = (a[:g.numel()] * g).sum()
    loss.backward()
    torch.cuda.synchronize()
    gpu = dict(a=a.detach().cpu().numpy(), dqfrc=q.grad.cpu().numpy(),
               daref=ar.grad.cpu().numpy(), dJ=J.grad.cpu().numpy(),
               status=np.zeros(w.n, np.int32), iters=np.zeros(w.n, np.int32))
    ref = oracle.solve_workload(w)
    res = parity.compare(w, gpu, ref, np.arange(w.n))
    assert not res["bad"], res["bad"][:3]


@pytest.mark.parametrize("keep_factor", [True, False])
def test_adjoint_memory_flat_in_iterations(cuda_device, keep_factor):
    w = W.franka(n=4096, seed=22)
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    g = torch.from_numpy(w.g).to(cuda_device)
    peaks, state_bytes = [], []
    for K in range(1, 11):
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        J = batch.J.clone().requires_grad_(True)
        a = csag.contact_solve(batch, J=J, max_iter=K, keep_factor=keep_factor)
        (a[:g.numel()] * g).sum().backward()
        torch.cuda.synchronize()
        peaks.append(torch.cuda.max_memory_allocated() - base)
        state_bytes.append(solver.alloc_state(batch, keep_factor).nbytes())
        del a, J
    assert len(set(state_bytes)) == 1
    assert max(peaks) == min(peaks), peaks


@pytest.mark.parametrize("make", [lambda: W.nv96(n=256, seed=23), lambda: W.nc256(n=64, seed=24)],
                         ids=["nv96", "nc256"])
def test_adjoint_memory_flat_in_iterations_cta_sizes(cuda_device, make):
    # the one-CTA-per-instance kernels (nv 96; 1024 rows): the same flat state
    w = make()
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    g = torch.from_numpy(w.g).to(cuda_device)
    peaks = []
    for K in range(1, 11):
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        J = batch.J.clone().requires_grad_(True)
        a = csag.contact_solve(batch, J=J, max_iter=K)
        (a[:g.numel()] * g).sum().backward()
        torch.cuda.synchronize()
        peaks.append(torch.cuda.max_memory_allocated() - base)
        del a, J
    assert max(peaks) == min(peaks), peaks
