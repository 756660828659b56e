"""``torch.autograd.Function`` around the solve: the backward pass is the IFT
adjoint of Eq. 17, never an unrolled solver trace.

Forward runs ``cs_solve_fwd`` and keeps only the adjoint state (a*, a_lo, the
active set and, by default, the Cholesky factor of H(a*)), whose size does not
depend on the number of Newton iterations.  Backward runs
``cs_solve_adjoint`` on grad_a and returns dL/dJ, dL/dqfrc and dL/daref; when
M or D requires grad it runs ``cs_solve_adjoint_theta`` instead and also
returns dL/dM (with respect to a symmetric M: -(w a^T + a w^T)/2) and dL/dD
(-(J w) . min(jar, 0)), the remaining parameter terms of Eq. 17.

With ``keep_factor=False`` the factor is not stored; the backward rebuilds it
from the stored active set (less memory, one extra factorisation).
"""
from __future__ import annotations

import torch

from . import solver


class ContactSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, batch: solver.DeviceBatch, M, J, qfrc, aref, D,
                tol=solver.DEFAULT_TOL, max_iter=solver.DEFAULT_MAX_ITER,
                keep_factor=True):
        b = batch.with_data(M=M.detach().contiguous(), J=J.detach().contiguous(),
                            qfrc=qfrc.detach().contiguous(),
                            aref=aref.detach().contiguous(), D=D.detach().contiguous())
        a, state = solver.solve_fwd(b, tol=tol, max_iter=max_iter,
                                    keep_factor=keep_factor)
        ctx.batch = b
        ctx.state = state
        ctx.tol = tol
        ctx.max_iter = max_iter
        ctx.save_for_backward(a)
        ctx.mark_non_differentiable()
        return a

    @staticmethod
    def backward(ctx, grad_a):
        (a,) = ctx.saved_tensors
        theta = ctx.needs_input_grad[1] or ctx.needs_input_grad[5]
        res = solver.solve_adjoint(ctx.batch, a, ctx.state, grad_a.contiguous(),
                                   tol=ctx.tol, max_iter=ctx.max_iter, theta=theta)
        dq, dr, dJ = res[:3]
        b = ctx.batch
        dJ = dJ[:b.J.numel()].view_as(b.J) if b.J.numel() else torch.zeros_like(b.J)
        dr = dr[:b.aref.numel()].view_as(b.aref) if b.aref.numel() else torch.zeros_like(b.aref)
        dq = dq[:b.qfrc.numel()].view_as(b.qfrc)
        dM = dD = None
        if theta:
            dM = res[3][:b.M.numel()].view_as(b.M) if ctx.needs_input_grad[1] else None
            if ctx.needs_input_grad[5]:
                dD = (res[4][:b.D.numel()].view_as(b.D) if b.D.numel()
                      else torch.zeros_like(b.D))
        return None, dM, dJ, dq, dr, dD, None, None, None


def contact_solve(batch: solver.DeviceBatch, M=None, J=None, qfrc=None, aref=None,
                  D=None, tol=solver.DEFAULT_TOL, max_iter=solver.DEFAULT_MAX_ITER,
                  keep_factor=True):
    """a* for the batch; differentiable w.r.t. M, J, qfrc, aref and D."""
    return ContactSolve.apply(batch, batch.M if M is None else M,
                              batch.J if J is None else J,
                              batch.qfrc if qfrc is None else qfrc,
                              batch.aref if aref is None else aref,
                              batch.D if D is None else D, tol, max_iter,
                              keep_factor)


class UnrolledContactSolve(torch.autograd.Function):
    """The comparison the paper makes (Section III-E): the same solve, but
    differentiated by a reverse sweep through the recorded trace of at most K
    Newton steps.  The saved state is the trace, whose size grows with K."""

    @staticmethod
    def forward(ctx, batch: solver.DeviceBatch, M, J, qfrc, aref, D, K=10,
                tol=solver.DEFAULT_TOL):
        b = batch.with_data(M=M.detach().contiguous(), J=J.detach().contiguous(),
                            qfrc=qfrc.detach().contiguous(),
                            aref=aref.detach().contiguous(), D=D.detach().contiguous())
        st = solver.unrolled_fwd(b, K, tol=tol)
        ctx.batch = b
        # the output goes through save_for_backward (an attribute holding it
        # would form a reference cycle with the graph)
        ctx.save_for_backward(st.a)
        ctx.trace = (st.trace, st.tmask, st.status, st.iters, st.K)
        ctx.tol = tol
        ctx.mark_non_differentiable()
        return st.a

    @staticmethod
    def backward(ctx, grad_a):
        b = ctx.batch
        (a,) = ctx.saved_tensors
        trace, tmask, status, iters, K = ctx.trace
        st = solver.UnrolledState(a=a, trace=trace, tmask=tmask, status=status, iters=iters,
                                  K=K)
        dq, dr, dJ, dM, dD = solver.unrolled_bwd(b, st, grad_a.contiguous(), tol=ctx.tol)
        ng = ctx.needs_input_grad
        shape = lambda x, ref: (x[:ref.numel()].view_as(ref) if ref.numel()
                                else torch.zeros_like(ref))
        return (None, shape(dM, b.M) if ng[1] else None, shape(dJ, b.J) if ng[2] else None,
                shape(dq, b.qfrc) if ng[3] else None, shape(dr, b.aref) if ng[4] else None,
                shape(dD, b.D) if ng[5] else None, None, None)


def contact_solve_unrolled(batch: solver.DeviceBatch, M=None, J=None, qfrc=None,
                           aref=None, D=None, K=10, tol=solver.DEFAULT_TOL):
    """a after at most K Newton steps, differentiated through its trace."""
    return UnrolledContactSolve.apply(batch, batch.M if M is None else M,
                                      batch.J if J is None else J,
                                      batch.qfrc if qfrc is None else qfrc,
                                      batch.aref if aref is None else aref,
                                      batch.D if D is None else D, K, tol)
