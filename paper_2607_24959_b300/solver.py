"""Python entry points over the C ABI (torch tensors in, torch tensors out).

Names follow the C ABI: ``solve_fwd``, ``solve_adjoint``, ``solve_fused``.
PyTorch only provides device memory and the current CUDA stream; every
numerical step runs in ``libcs_b300.so``.
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np
import torch

from . import _lib

DEFAULT_TOL = 1e-8
DEFAULT_MAX_ITER = 50


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@dataclasses.dataclass
class DeviceBatch:
    """A packed ragged batch resident on one GPU (layout of cs_batch)."""

    inst: torch.Tensor     # uint8 view of the cs_inst table (40 B / instance)
    M: torch.Tensor
    J: torch.Tensor
    qfrc: torch.Tensor
    aref: torch.Tensor
    D: torch.Tensor
    n: int
    nv_max: int
    m_max: int
    inst_host: np.ndarray  # the same table on the host

    @classmethod
    def from_workload(cls, w, device="cuda"):
        dev = torch.device(device)
        f = lambda x: torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(dev)
        inst = torch.from_numpy(np.ascontiguousarray(w.inst).view(np.uint8)).to(dev)
        return cls(inst, f(w.M), f(w.J), f(w.qfrc), f(w.aref), f(w.D), w.n,
                   max(w.nv_max, 1), w.m_max, np.ascontiguousarray(w.inst))

    def with_data(self, M=None, J=None, qfrc=None, aref=None, D=None):
        """Same layout, other data tensors (used by the autograd wrapper)."""
        return dataclasses.replace(
            self, M=self.M if M is None else M, J=self.J if J is None else J,
            qfrc=self.qfrc if qfrc is None else qfrc,
            aref=self.aref if aref is None else aref, D=self.D if D is None else D)

    @property
    def total_v(self):
        return self.qfrc.numel()

    @property
    def total_r(self):
        return self.aref.numel()

    def cstruct(self) -> _lib.CsBatch:
        for t in (self.M, self.J, self.qfrc, self.aref, self.D):
            if t.dtype != torch.float32 or not t.is_contiguous() or not t.is_cuda:
                raise ValueError("batch data must be contiguous float32 CUDA tensors")
        b = _lib.CsBatch()
        b.n = self.n
        b.nv_max = self.nv_max
        b.m_max = self.m_max
        b.inst = self.inst.data_ptr()
        b.M = self.M.data_ptr()
        b.J = self.J.data_ptr() if self.J.numel() else self.M.data_ptr()
        b.qfrc = self.qfrc.data_ptr()
        b.aref = self.aref.data_ptr() if self.aref.numel() else self.qfrc.data_ptr()
        b.D = self.D.data_ptr() if self.D.numel() else self.qfrc.data_ptr()
        b.total_M = self.M.numel()
        b.total_J = self.J.numel()
        b.total_v = self.qfrc.numel()
        b.total_r = self.aref.numel()
        return b


def options(tol=DEFAULT_TOL, max_iter=DEFAULT_MAX_ITER, keep_factor=True,
            warps_per_block=0) -> _lib.CsOptions:
    o = _lib.CsOptions()
    o.tol = float(tol)
    o.max_iter = int(max_iter)
    o.keep_factor = 1 if keep_factor else 0
    o.warps_per_block = int(warps_per_block)
    return o


@dataclasses.dataclass
class State:
    """Adjoint state of cs_solve_fwd (device tensors); size independent of K."""

    a_lo: torch.Tensor
    act: torch.Tensor
    L: torch.Tensor | None
    status: torch.Tensor
    iters: torch.Tensor
    keep_factor: bool

    def cstruct(self) -> _lib.CsState:
        s = _lib.CsState()
        s.a_lo = self.a_lo.data_ptr()
        s.act = self.act.data_ptr()
        s.L = self.L.data_ptr() if self.L is not None else None
        s.status = self.status.data_ptr()
        s.iters = self.iters.data_ptr()
        return s

    def nbytes(self) -> int:
        return sum(t.numel() * t.element_size()
                   for t in (self.a_lo, self.act, self.L, self.status, self.iters)
                   if t is not None)


def alloc_state(batch: DeviceBatch, keep_factor=True) -> State:
    dev = batch.M.device
    return State(
        a_lo=torch.empty(max(batch.total_v, 1), dtype=torch.float32, device=dev),
        act=torch.empty(max(batch.total_r, 1), dtype=torch.uint8, device=dev),
        L=(torch.empty(max(batch.M.numel(), 1), dtype=torch.float32, device=dev)
           if keep_factor else None),
        status=torch.empty(max(batch.n, 1), dtype=torch.int32, device=dev),
        iters=torch.empty(max(batch.n, 1), dtype=torch.int32, device=dev),
        keep_factor=bool(keep_factor))


def solve_fwd(batch: DeviceBatch, tol=DEFAULT_TOL, max_iter=DEFAULT_MAX_ITER,
              keep_factor=True, warps_per_block=0, a=None, state=None):
    """Forward solve; returns (a, state)."""
    lib = _lib.load()
    dev = batch.M.device
    if a is None:
        a = torch.empty(max(batch.total_v, 1), dtype=torch.float32, device=dev)
    if state is None:
        state = alloc_state(batch, keep_factor)
    b = batch.cstruct()
    o = options(tol, max_iter, keep_factor, warps_per_block)
    st = state.cstruct()
    _lib.check(lib.cs_solve_fwd(ctypes.byref(b), ctypes.byref(o), _ptr(a),
                                ctypes.byref(st), _stream()), "cs_solve_fwd")
    return a, state


class OwnedState:
    """A forward state allocated and owned by the library (cs_solve_fwd_alloc /
    cs_state_create); usable wherever a State is, freed by close()."""

    def __init__(self, ptr, n: int, device):
        self._ptr = ptr
        self.n = n
        self.device = device
        self.keep_factor = bool(ptr.contents.L)

    def cstruct(self) -> _lib.CsState:
        return self._ptr.contents

    def status_iters(self):
        """Per-instance status and Newton step counts (cs_state_status)."""
        st = torch.empty(max(self.n, 1), dtype=torch.int32, device=self.device)
        it = torch.empty(max(self.n, 1), dtype=torch.int32, device=self.device)
        _lib.check(_lib.load().cs_state_status(self._ptr, _ptr(st), _ptr(it), _stream()),
                   "cs_state_status")
        return st[:self.n], it[:self.n]

    def close(self):
        if self._ptr:
            torch.cuda.synchronize(self.device)
            _lib.load().cs_state_free(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_fwd_owned(batch: DeviceBatch, tol=DEFAULT_TOL, max_iter=DEFAULT_MAX_ITER,
                    keep_factor=True, warps_per_block=0, a=None, state: OwnedState | None = None):
    """Forward solve into a library-owned state (cs_solve_fwd_alloc); returns
    (a, OwnedState).  A state from an earlier call on a batch of the same
    sizes is reused when given."""
    lib = _lib.load()
    dev = batch.M.device
    if a is None:
        a = torch.empty(max(batch.total_v, 1), dtype=torch.float32, device=dev)
    b = batch.cstruct()
    o = options(tol, max_iter, keep_factor, warps_per_block)
    ptr = state._ptr if state is not None else ctypes.POINTER(_lib.CsState)()
    _lib.check(lib.cs_solve_fwd_alloc(ctypes.byref(b), ctypes.byref(o), _ptr(a),
                                      ctypes.byref(ptr), _stream()), "cs_solve_fwd_alloc")
    if state is None:
        state = OwnedState(ptr, batch.n, dev)
    return a, state


def solve_adjoint(batch: DeviceBatch, a, state: State, g, tol=DEFAULT_TOL,
                  max_iter=DEFAULT_MAX_ITER, warps_per_block=0, out=None, theta=False):
    """IFT adjoint at the forward state; returns (dqfrc, daref, dJ), or with
    ``theta`` (dqfrc, daref, dJ, dM, dD) from cs_solve_adjoint_theta (dM packed
    like M, dD like D)."""
    lib = _lib.load()
    dev = batch.M.device
    if out is None:
        out = (torch.empty(max(batch.total_v, 1), dtype=torch.float32, device=dev),
               torch.empty(max(batch.total_r, 1), dtype=torch.float32, device=dev),
               torch.empty(max(batch.J.numel(), 1), dtype=torch.float32, device=dev))
        if theta:
            out = out + (torch.empty(max(batch.M.numel(), 1), dtype=torch.float32, device=dev),
                         torch.empty(max(batch.total_r, 1), dtype=torch.float32, device=dev))
    b = batch.cstruct()
    o = options(tol, max_iter, state.keep_factor, warps_per_block)
    st = state.cstruct()
    g = g.contiguous()
    if theta:
        dq, dr, dJ, dM, dD = out
        _lib.check(lib.cs_solve_adjoint_theta(
            ctypes.byref(b), ctypes.byref(o), _ptr(a), ctypes.byref(st), _ptr(g), _ptr(dq),
            _ptr(dr), _ptr(dJ), _ptr(dM), _ptr(dD), _stream()), "cs_solve_adjoint_theta")
        return dq, dr, dJ, dM, dD
    dq, dr, dJ = out[:3]
    _lib.check(lib.cs_solve_adjoint(ctypes.byref(b), ctypes.byref(o), _ptr(a),
                                    ctypes.byref(st), _ptr(g), _ptr(dq), _ptr(dr),
                                    _ptr(dJ), _stream()), "cs_solve_adjoint")
    return dq, dr, dJ


@dataclasses.dataclass
class UnrolledState:
    """What the unrolled reverse sweep needs: the trace of the executed K
    steps (grows linearly with K), the returned a, status and step counts."""

    a: torch.Tensor
    trace: torch.Tensor
    tmask: torch.Tensor
    status: torch.Tensor
    iters: torch.Tensor
    K: int

    def nbytes(self) -> int:
        """Bytes kept between the forward and the reverse sweep (a excluded,
        as for State)."""
        return sum(t.numel() * t.element_size()
                   for t in (self.trace, self.tmask, self.status, self.iters))


def unrolled_fwd(batch: DeviceBatch, K: int, tol=DEFAULT_TOL) -> UnrolledState:
    """At most K Newton steps with their trace recorded (cs_unrolled_fwd)."""
    lib = _lib.load()
    dev = batch.M.device
    b = batch.cstruct()
    nf = int(lib.cs_unrolled_trace_floats(ctypes.byref(b), int(K)))
    nm = int(lib.cs_unrolled_mask_bytes(ctypes.byref(b), int(K)))
    st = UnrolledState(
        a=torch.empty(max(batch.total_v, 1), dtype=torch.float32, device=dev),
        trace=torch.empty(max(nf, 1), dtype=torch.float32, device=dev),
        tmask=torch.empty(max(nm, 1), dtype=torch.uint8, device=dev),
        status=torch.empty(max(batch.n, 1), dtype=torch.int32, device=dev),
        iters=torch.empty(max(batch.n, 1), dtype=torch.int32, device=dev), K=int(K))
    o = options(tol, K, False, 0)
    _lib.check(lib.cs_unrolled_fwd(ctypes.byref(b), ctypes.byref(o), _ptr(st.a),
                                   _ptr(st.trace), _ptr(st.tmask), _ptr(st.status),
                                   _ptr(st.iters), _stream()), "cs_unrolled_fwd")
    return st


def unrolled_bwd(batch: DeviceBatch, st: UnrolledState, g, tol=DEFAULT_TOL):
    """Reverse sweep through the recorded steps (cs_unrolled_bwd); returns
    (dqfrc, daref, dJ, dM, dD) packed like qfrc, aref, J, M and D."""
    lib = _lib.load()
    dev = batch.M.device
    dq = torch.empty(max(batch.total_v, 1), dtype=torch.float32, device=dev)
    dr = torch.empty(max(batch.total_r, 1), dtype=torch.float32, device=dev)
    dJ = torch.empty(max(batch.J.numel(), 1), dtype=torch.float32, device=dev)
    dM = torch.empty(max(batch.M.numel(), 1), dtype=torch.float32, device=dev)
    dD = torch.empty(max(batch.total_r, 1), dtype=torch.float32, device=dev)
    b = batch.cstruct()
    o = options(tol, st.K, False, 0)
    g = g.contiguous()
    _lib.check(lib.cs_unrolled_bwd(ctypes.byref(b), ctypes.byref(o), _ptr(st.a),
                                   _ptr(st.trace), _ptr(st.tmask), _ptr(st.status),
                                   _ptr(st.iters), _ptr(g), _ptr(dq), _ptr(dr), _ptr(dJ),
                                   _ptr(dM), _ptr(dD), _stream()), "cs_unrolled_bwd")
    return dq, dr, dJ, dM, dD


def fused_workspace_bytes(n: int) -> int:
    return int(_lib.load().cs_fused_workspace_bytes(int(n)))


@dataclasses.dataclass
class FusedOut:
    a: torch.Tensor
    dqfrc: torch.Tensor
    daref: torch.Tensor
    dJ: torch.Tensor
    status: torch.Tensor
    iters: torch.Tensor
    workspace: torch.Tensor
    dM: torch.Tensor | None = None   # dL/dM (symmetric M), packed like M
    dD: torch.Tensor | None = None   # dL/dD, packed like D


def alloc_fused(batch: DeviceBatch, theta: bool = False) -> FusedOut:
    dev = batch.M.device
    ws = torch.zeros(fused_workspace_bytes(batch.n), dtype=torch.uint8, device=dev)
    return FusedOut(
        a=torch.empty(max(batch.total_v, 1), dtype=torch.float32, device=dev),
        dqfrc=torch.empty(max(batch.total_v, 1), dtype=torch.float32, device=dev),
        daref=torch.empty(max(batch.total_r, 1), dtype=torch.float32, device=dev),
        dJ=torch.empty(max(batch.J.numel(), 1), dtype=torch.float32, device=dev),
        status=torch.empty(max(batch.n, 1), dtype=torch.int32, device=dev),
        iters=torch.empty(max(batch.n, 1), dtype=torch.int32, device=dev),
        workspace=ws,
        dM=(torch.empty(max(batch.M.numel(), 1), dtype=torch.float32, device=dev)
            if theta else None),
        dD=(torch.empty(max(batch.total_r, 1), dtype=torch.float32, device=dev)
            if theta else None))


def solve_fused(batch: DeviceBatch, g, order=None, tol=DEFAULT_TOL,
                max_iter=DEFAULT_MAX_ITER, warps_per_block=0, out: FusedOut | None = None,
                theta: bool = False):
    """Fused forward + adjoint in one persistent launch; returns FusedOut.
    With ``theta`` (or an ``out`` holding dM/dD) the launch also writes dL/dM
    and dL/dD (cs_solve_fused_theta)."""
    lib = _lib.load()
    if out is None:
        out = alloc_fused(batch, theta)
    b = batch.cstruct()
    o = options(tol, max_iter, True, warps_per_block)
    g = g.contiguous()
    if out.dM is not None or out.dD is not None:
        _lib.check(lib.cs_solve_fused_theta(
            ctypes.byref(b), ctypes.byref(o), _ptr(g), _ptr(order), _ptr(out.a),
            _ptr(out.dqfrc), _ptr(out.daref), _ptr(out.dJ), _ptr(out.dM), _ptr(out.dD),
            _ptr(out.status), _ptr(out.iters), _ptr(out.workspace), out.workspace.numel(),
            _stream()), "cs_solve_fused_theta")
        return out
    _lib.check(lib.cs_solve_fused(
        ctypes.byref(b), ctypes.byref(o), _ptr(g), _ptr(order), _ptr(out.a),
        _ptr(out.dqfrc), _ptr(out.daref), _ptr(out.dJ), _ptr(out.status),
        _ptr(out.iters), _ptr(out.workspace), out.workspace.numel(), _stream()),
        "cs_solve_fused")
    return out


NCG_MAX_ITER = 5000   # conjugate-gradient steps (Newton needs about ten)


def solve_fused_ncg(batch: DeviceBatch, g, order=None, tol=DEFAULT_TOL, max_iter=NCG_MAX_ITER,
                    warps_per_block=0, out: FusedOut | None = None) -> FusedOut:
    """Fused forward + adjoint with the nonlinear conjugate-gradient forward
    solver (cs_solve_fused_ncg); the adjoint is the same IFT rule."""
    lib = _lib.load()
    if out is None:
        out = alloc_fused(batch)
    b = batch.cstruct()
    o = options(tol, max_iter, True, warps_per_block)
    g = g.contiguous()
    _lib.check(lib.cs_solve_fused_ncg(
        ctypes.byref(b), ctypes.byref(o), _ptr(g), _ptr(order), _ptr(out.a), _ptr(out.dqfrc),
        _ptr(out.daref), _ptr(out.dJ), _ptr(out.status), _ptr(out.iters), _ptr(out.workspace),
        out.workspace.numel(), _stream()), "cs_solve_fused_ncg")
    return out


@dataclasses.dataclass
class EllipticOut:
    """Outputs of the round-cone fused solve (packed like the batch)."""

    fused: FusedOut        # a, dqfrc, daref, dJ, status, iters, workspace, dM, dD
    dmu: torch.Tensor


ELLIPTIC_MAX_ITER = 100   # the round cone's middle zone needs more Newton steps


def solve_fused_elliptic(batch: DeviceBatch, g, mu, order=None, tol=DEFAULT_TOL,
                         max_iter=ELLIPTIC_MAX_ITER, warps_per_block=0,
                         out: EllipticOut | None = None) -> EllipticOut:
    """Fused forward + adjoint with the round Coulomb cone
    (cs_solve_fused_elliptic): three rows per contact, mu per contact on its
    normal row; writes every parameter gradient including dM, dD and dmu."""
    lib = _lib.load()
    if out is None:
        out = EllipticOut(alloc_fused(batch, theta=True),
                          torch.empty(max(batch.total_r, 1), dtype=torch.float32,
                                      device=batch.M.device))
    f = out.fused
    b = batch.cstruct()
    o = options(tol, max_iter, True, warps_per_block)
    g = g.contiguous()
    mu = mu.contiguous()
    _lib.check(lib.cs_solve_fused_elliptic(
        ctypes.byref(b), ctypes.byref(o), _ptr(mu), _ptr(g), _ptr(order), _ptr(f.a),
        _ptr(f.dqfrc), _ptr(f.daref), _ptr(f.dJ), _ptr(f.dM), _ptr(f.dD), _ptr(out.dmu),
        _ptr(f.status), _ptr(f.iters), _ptr(f.workspace), f.workspace.numel(), _stream()),
        "cs_solve_fused_elliptic")
    return out


def solve_fused_static(batch: DeviceBatch, g, tol=DEFAULT_TOL, max_iter=DEFAULT_MAX_ITER,
                       warps_per_block=0, cost_ordered=True, out: FusedOut | None = None):
    """solve_fused without any device allocation by the library: the claim
    counter and order live in the library's static device array
    (cs_solve_fused_static).  ``out`` may be preallocated by the caller (its
    workspace field is not used)."""
    lib = _lib.load()
    if out is None:
        out = alloc_fused(batch)
    b = batch.cstruct()
    o = options(tol, max_iter, True, warps_per_block)
    g = g.contiguous()
    inst = np.ascontiguousarray(batch.inst_host) if cost_ordered else None
    _lib.check(lib.cs_solve_fused_static(
        ctypes.byref(b), ctypes.byref(o), _ptr(g),
        None if inst is None else inst.ctypes.data_as(ctypes.c_void_p), _ptr(out.a),
        _ptr(out.dqfrc), _ptr(out.daref), _ptr(out.dJ), _ptr(out.status), _ptr(out.iters),
        _stream()), "cs_solve_fused_static")
    return out


def cost_order(inst_host: np.ndarray) -> np.ndarray:
    """Claim order for the persistent kernel: most expensive instances first.

    Cost model per instance: m*nv^2 + nv^3 (the Newton-matrix assembly and the
    Cholesky factor dominate an iteration)."""
    nv = inst_host["nv"].astype(np.int64)
    m = inst_host["m"].astype(np.int64)
    cost = m * nv * nv + nv ** 3
    return np.argsort(-cost, kind="stable").astype(np.int32)


class FusedPlan:
    """cs_plan for the fused path on one batch: per-(nv, m) bucket kernels,
    cost-ordered claims, autotuned warps per block, one CUDA graph.

    The plan keeps references to the batch, g and the output tensors it was
    made for; ``launch()`` re-runs the whole fused solve on them.
    """

    def __init__(self, batch: DeviceBatch, g, tol=DEFAULT_TOL, max_iter=DEFAULT_MAX_ITER,
                 autotune=True, graph=True, warps_per_block=0, out: FusedOut | None = None,
                 theta: bool = False):
        lib = _lib.load()
        self.batch = batch
        self.g = g.contiguous()
        self.out = out if out is not None else alloc_fused(batch, theta)
        self._b = batch.cstruct()
        self._o = options(tol, max_iter, True, warps_per_block)
        self._inst_host = np.ascontiguousarray(batch.inst_host)
        flags = ((_lib.CS_PLAN_AUTOTUNE if autotune else 0) |
                 (_lib.CS_PLAN_GRAPH if graph else 0))
        h = ctypes.c_void_p(None)
        o = self.out
        if o.dM is not None or o.dD is not None:
            _lib.check(lib.cs_plan_create_fused_theta(
                ctypes.byref(self._b), ctypes.byref(self._o),
                self._inst_host.ctypes.data_as(ctypes.c_void_p), _ptr(self.g), _ptr(o.a),
                _ptr(o.dqfrc), _ptr(o.daref), _ptr(o.dJ), _ptr(o.dM), _ptr(o.dD),
                _ptr(o.status), _ptr(o.iters), flags, _stream(), ctypes.byref(h)),
                "cs_plan_create_fused_theta")
        else:
            _lib.check(lib.cs_plan_create_fused(
                ctypes.byref(self._b), ctypes.byref(self._o),
                self._inst_host.ctypes.data_as(ctypes.c_void_p), _ptr(self.g), _ptr(o.a),
                _ptr(o.dqfrc), _ptr(o.daref), _ptr(o.dJ), _ptr(o.status), _ptr(o.iters),
                flags, _stream(), ctypes.byref(h)), "cs_plan_create_fused")
        self._h = h
        self._lib = lib

    def launch(self):
        _lib.check(self._lib.cs_plan_launch(self._h, _stream()), "cs_plan_launch")
        return self.out

    def describe(self) -> dict:
        info = _lib.CsPlanInfo()
        _lib.check(self._lib.cs_plan_describe(self._h, ctypes.byref(info)), "cs_plan_describe")
        k = info.n_kernels
        return {"kernels": k, "graph": bool(info.graph),
                "buckets": [{"nv_bucket": info.nv_bucket[i], "rows_per_lane": info.rows_per_lane[i],
                             "instances": info.instances[i],
                             "warps_per_block": info.warps_per_block[i],
                             "kernel": "cta" if info.cta[i] else "warp",
                             "tuned_ms": round(float(info.tuned_ms[i]), 4)}
                            for i in range(k)]}

    def close(self):
        if getattr(self, "_h", None):
            torch.cuda.synchronize()
            self._lib.cs_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune_cache_dump() -> str:
    lib = _lib.load()
    n = lib.cs_autotune_cache_dump(None, 0)
    buf = ctypes.create_string_buffer(n + 1)
    lib.cs_autotune_cache_dump(buf, n + 1)
    return buf.value.decode()


def autotune_cache_load(text: str) -> int:
    return int(_lib.load().cs_autotune_cache_load(text.encode()))


class HostPipeline:
    """Fused solve of a host-resident batch with copies and compute overlapped.

    The batch (pinned host arrays in the packed layout) is cut into
    ``chunks`` contiguous instance ranges; their blocks are contiguous in
    every packed array, so each chunk is one slice per array.  Per step and
    chunk: the upload stream copies the chunk's inputs (instance table
    included) into full-size device arrays at the same offsets, the compute
    stream runs the chunk's plan (its own bucket kernels and CUDA graph), the
    download stream copies the chunk's outputs back.  Uploads of chunk c+1,
    the solve of chunk c and the download of chunk c-1 overlap.  Events make
    a chunk's buffers safe to reuse across steps.
    """

    def __init__(self, w, chunks=8, device="cuda", tol=DEFAULT_TOL, max_iter=DEFAULT_MAX_ITER,
                 autotune=False):
        dev = torch.device(device)
        pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
        self.w = w
        self.h_in = dict(inst=pin(np.ascontiguousarray(w.inst).view(np.uint8)), M=pin(w.M),
                         J=pin(w.J), qfrc=pin(w.qfrc), aref=pin(w.aref), D=pin(w.D), g=pin(w.g))
        self.d_in = {k: torch.empty_like(v, device=dev) for k, v in self.h_in.items()}
        full = DeviceBatch(self.d_in["inst"], self.d_in["M"], self.d_in["J"], self.d_in["qfrc"],
                           self.d_in["aref"], self.d_in["D"], w.n, max(w.nv_max, 1), w.m_max,
                           np.ascontiguousarray(w.inst))
        self.out = alloc_fused(full)
        self.h_out = dict(a=torch.empty_like(self.out.a, device="cpu").pin_memory(),
                          dqfrc=torch.empty_like(self.out.dqfrc, device="cpu").pin_memory(),
                          daref=torch.empty_like(self.out.daref, device="cpu").pin_memory(),
                          dJ=torch.empty_like(self.out.dJ, device="cpu").pin_memory(),
                          status=torch.empty_like(self.out.status, device="cpu").pin_memory(),
                          iters=torch.empty_like(self.out.iters, device="cpu").pin_memory())
        n = w.n
        bounds = np.linspace(0, n, min(chunks, max(n, 1)) + 1).astype(int)
        inst = w.inst
        self.chunks = []
        for c0, c1 in zip(bounds[:-1], bounds[1:]):
            if c1 <= c0:
                continue
            e0, e1 = inst[c0], inst[c1 - 1]
            sl = dict(
                inst=(c0 * 40, c1 * 40),
                M=(int(e0["off_M"]), int(e1["off_M"]) + int(e1["nv"]) ** 2),
                J=(int(e0["off_J"]), int(e1["off_J"]) + int(e1["m"]) * int(e1["nv"])),
                v=(int(e0["off_v"]), int(e1["off_v"]) + int(e1["nv"])),
                r=(int(e0["off_r"]), int(e1["off_r"]) + int(e1["m"])))
            part = DeviceBatch(self.d_in["inst"][c0 * 40:c1 * 40], full.M, full.J, full.qfrc,
                               full.aref, full.D, int(c1 - c0),
                               max(1, int(inst["nv"][c0:c1].max())), int(inst["m"][c0:c1].max()),
                               np.ascontiguousarray(inst[c0:c1]))
            self.chunks.append(dict(range=(int(c0), int(c1)), sl=sl, batch=part))
        self.s_in = torch.cuda.Stream(device=dev)
        self.s_comp = torch.cuda.Stream(device=dev)
        self.s_out = torch.cuda.Stream(device=dev)
        # plans read the inputs already uploaded: upload once before planning
        for k in self.d_in:
            self.d_in[k].copy_(self.h_in[k])
        torch.cuda.synchronize()
        with torch.cuda.stream(self.s_comp):
            for ch in self.chunks:
                c0, c1 = ch["range"]
                # per-instance outputs (status, iters) are indexed by the
                # instance's position in its chunk
                o = FusedOut(self.out.a, self.out.dqfrc, self.out.daref, self.out.dJ,
                             self.out.status[c0:c1], self.out.iters[c0:c1], self.out.workspace)
                ch["plan"] = FusedPlan(ch["batch"], self.d_in["g"], tol=tol, max_iter=max_iter,
                                       autotune=autotune, graph=True, out=o)
        torch.cuda.synchronize()
        mk = lambda: torch.cuda.Event()
        for ch in self.chunks:
            ch["ev_in"], ch["ev_comp"], ch["ev_out"] = mk(), mk(), mk()
            ch["ev_comp"].record(self.s_comp)
            ch["ev_out"].record(self.s_out)

    def _copy(self, dst, src, lo, hi):
        if hi > lo:
            dst[lo:hi].copy_(src[lo:hi], non_blocking=True)

    def step(self):
        """Enqueue one pipelined pass (host inputs -> solve -> host outputs)."""
        for ch in self.chunks:
            sl = ch["sl"]
            with torch.cuda.stream(self.s_in):
                self.s_in.wait_event(ch["ev_comp"])       # inputs no longer read
                self._copy(self.d_in["inst"], self.h_in["inst"], *sl["inst"])
                self._copy(self.d_in["M"], self.h_in["M"], *sl["M"])
                self._copy(self.d_in["J"], self.h_in["J"], *sl["J"])
                for k in ("qfrc", "g"):
                    self._copy(self.d_in[k], self.h_in[k], *sl["v"])
                for k in ("aref", "D"):
                    self._copy(self.d_in[k], self.h_in[k], *sl["r"])
                ch["ev_in"].record(self.s_in)
            with torch.cuda.stream(self.s_comp):
                self.s_comp.wait_event(ch["ev_in"])
                self.s_comp.wait_event(ch["ev_out"])      # outputs already read back
                ch["plan"].launch()
                ch["ev_comp"].record(self.s_comp)
            with torch.cuda.stream(self.s_out):
                self.s_out.wait_event(ch["ev_comp"])
                c0, c1 = ch["range"]
                self._copy(self.h_out["a"], self.out.a, *sl["v"])
                self._copy(self.h_out["dqfrc"], self.out.dqfrc, *sl["v"])
                self._copy(self.h_out["daref"], self.out.daref, *sl["r"])
                self._copy(self.h_out["dJ"], self.out.dJ, *sl["J"])
                self._copy(self.h_out["status"], self.out.status, c0, c1)
                self._copy(self.h_out["iters"], self.out.iters, c0, c1)
                ch["ev_out"].record(self.s_out)

    def bytes_per_step(self):
        h2d = sum(v.numel() * v.element_size() for v in self.h_in.values())
        d2h = sum(v.numel() * v.element_size() for v in self.h_out.values())
        return h2d, d2h

    def close(self):
        torch.cuda.synchronize()
        for ch in self.chunks:
            ch["plan"].close()
