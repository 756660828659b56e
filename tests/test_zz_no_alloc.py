"""cs_solve_fused_static: the fused solve for callers that cannot allocate
device memory (its scratch lives in a static device array of the library).

It must give the results of cs_solve_fused (which takes a caller workspace)
within the parity tolerances, on two calls in a row (the second call reuses
the array the first one left behind), and refuse batches beyond the array's
capacity before touching the GPU.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2607_24959_b300 import _lib, solver, workloads as W
from tests import parity


def _outputs(out):
    torch.cuda.synchronize()
    return dict(a=out.a.cpu().numpy(), dqfrc=out.dqfrc.cpu().numpy(),
                daref=out.daref.cpu().numpy(), dJ=out.dJ.cpu().numpy(),
                status=out.status.cpu().numpy(), iters=out.iters.cpu().numpy())


def _close(w, got, ref):
    for b in range(w.n):
        e = w.inst[b]
        nv, m = int(e["nv"]), int(e["m"])
        ov, orr, oJ = int(e["off_v"]), int(e["off_r"]), int(e["off_J"])
        assert got["status"][b] == ref["status"][b]
        assert parity.rel(got["a"][ov:ov + nv], ref["a"][ov:ov + nv]) <= parity.A_TOL
        assert parity.rel(got["dqfrc"][ov:ov + nv], ref["dqfrc"][ov:ov + nv]) <= parity.G_TOL
        if m:
            assert parity.rel(got["daref"][orr:orr + m], ref["daref"][orr:orr + m]) <= parity.G_TOL
            assert parity.rel(got["dJ"][oJ:oJ + m * nv], ref["dJ"][oJ:oJ + m * nv]) <= parity.G_TOL


def _batch_with_cta_instances():
    """Quadruped instances (one warp each) and nv = 96 instances (one CTA
    each, as in the scaling-extremes workload) in one batch."""
    parts = [W.quadruped(n=400, seed=99).instance(b) for b in range(400)]
    big = W.generate("nv96-mix", 12, 96, 16, seed=98, cond=1e4)
    parts += [big.instance(b) for b in range(big.n)]
    return W.pack(parts, name="warp+cta")


@pytest.mark.gpu
@pytest.mark.parametrize("mixed", [False, True])
def test_static_scratch_matches_workspace_path_twice(cuda_device, mixed):
    w = _batch_with_cta_instances() if mixed else W.quadruped(n=2500, seed=99)
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    g = torch.from_numpy(w.g).to(cuda_device)
    ref = _outputs(solver.solve_fused(batch, g))
    out = solver.alloc_fused(batch)          # outputs preallocated by the caller
    # the first call in a fresh process may load the library's module that
    # holds the static array (the runtime's lazy module loading), which is
    # where the array's memory comes from; it is checked like the others
    _close(w, _outputs(solver.solve_fused_static(batch, g, out=out)), ref)
    free0 = torch.cuda.mem_get_info(cuda_device)[0]
    # two calls in a row: cost-ordered claims, then index-order claims that
    # reuse the counter and order left in the static array by the first call
    for ordered in (True, False):
        got = _outputs(solver.solve_fused_static(batch, g, cost_ordered=ordered, out=out))
        # the calls allocate no device memory
        assert torch.cuda.mem_get_info(cuda_device)[0] == free0
        _close(w, got, ref)


def test_static_scratch_rejects_oversized_batches():
    lib = _lib.load()
    b = _lib.CsBatch()
    b.n, b.nv_max, b.m_max = _lib.STATIC_MAX_INSTANCES + 1, 18, 128
    b.inst = b.M = b.J = b.qfrc = b.aref = b.D = 0x10000
    b.total_M = b.total_J = b.total_v = b.total_r = 1 << 30
    o = solver.options()
    f = ctypes.c_void_p(0x30000)
    rc = lib.cs_solve_fused_static(ctypes.byref(b), ctypes.byref(o), f, None, f, f, f, f, f, f,
                                   None)
    assert rc == _lib.CS_EUNSUPPORTED
    assert b"static scratch capacity" in lib.cs_last_error()
