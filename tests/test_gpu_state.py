"""The library-owned adjoint state (cs_solve_fwd_alloc, cs_state_status,
cs_state_free) runs the same kernels as a caller-owned cs_state: same a,
statuses, step counts and gradients, bit for bit."""
import numpy as np
import pytest
import torch

from paper_2607_24959_b300 import solver, workloads as W
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("keep_factor", [True, False])
def test_owned_state_equals_caller_state(cuda_device, keep_factor):
    w = W.quadruped(n=600, seed=91)
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    g = torch.from_numpy(w.g).to(cuda_device)
    a1, s1 = solver.solve_fwd(batch, keep_factor=keep_factor)
    a2, s2 = solver.solve_fwd_owned(batch, keep_factor=keep_factor)
    assert s2.keep_factor == keep_factor
    st, it = s2.status_iters()
    torch.cuda.synchronize()
    masks = parity.valid_mask(w)

    def same(x, y, key):       # the real entries (padding between blocks is not written)
        return np.array_equal(parity.valid(w, {key: x.cpu().numpy()}, key, masks),
                              parity.valid(w, {key: y.cpu().numpy()}, key, masks))

    assert same(a1, a2, "a")
    assert torch.equal(st, s1.status[:w.n]) and torch.equal(it, s1.iters[:w.n])
    assert int(st.max()) == 0
    g1 = solver.solve_adjoint(batch, a1, s1, g)
    g2 = solver.solve_adjoint(batch, a2, s2, g)
    torch.cuda.synchronize()
    for x, y, key in zip(g1, g2, ("dqfrc", "daref", "dJ")):
        assert same(x, y, key), key
    # the state is reused by a second forward on a batch of the same sizes
    a3, s3 = solver.solve_fwd_owned(batch, keep_factor=keep_factor, state=s2)
    torch.cuda.synchronize()
    assert s3 is s2 and same(a3, a1, "a")
    # checked against the oracle like any other forward + adjoint
    res = dict(a=a2.cpu().numpy(), dqfrc=g2[0].cpu().numpy(), daref=g2[1].cpu().numpy(),
               dJ=g2[2].cpu().numpy(), status=st.cpu().numpy(), iters=it.cpu().numpy())
    import oracle
    ref = oracle.solve_workload(w, threads=8)
    out = parity.compare(w, res, ref, np.arange(w.n))
    assert not out["bad"], out["worst"]
    s2.close()
