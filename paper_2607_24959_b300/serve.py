"""Serving binding: continuous batching of contact solves (cs_serve_*).

Each request is one instance (host numpy arrays) solved forward and
differentiated with its own g; ``submit`` copies the data and returns a
ticket, ``poll`` returns the result once its batch has come back.  Batching,
admission by device memory, streams and transfers all happen in the
library's native scheduler thread.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from .solver import DEFAULT_MAX_ITER, DEFAULT_TOL


def _f32(x):
    return np.ascontiguousarray(np.asarray(x, np.float32))


class Server:
    def __init__(self, arena_bytes=1 << 30, streams=4, max_batch=4096, policy="continuous",
                 fixed_batch=1024, tol=DEFAULT_TOL, max_iter=DEFAULT_MAX_ITER, max_queue=0,
                 queue_timeout_ms=0):
        self._lib = _lib.load()
        c = _lib.CsServeConfig()
        c.arena_bytes = int(arena_bytes)
        c.streams = int(streams)
        c.max_batch = int(max_batch)
        c.policy = _lib.CS_SERVE_FIXED if policy == "fixed" else _lib.CS_SERVE_CONTINUOUS
        c.fixed_batch = int(fixed_batch)
        c.tol = float(tol)
        c.max_iter = int(max_iter)
        c.max_queue = int(max_queue)
        c.queue_timeout_ms = int(queue_timeout_ms)
        h = ctypes.c_void_p(None)
        _lib.check(self._lib.cs_serve_create(ctypes.byref(c), ctypes.byref(h)), "cs_serve_create")
        self._h = h
        self._shapes = {}

    def submit(self, M, J, qfrc, aref, D, g) -> int:
        M, J, q, ar, D, g = (_f32(x) for x in (M, J, qfrc, aref, D, g))
        nv = M.shape[0]
        m = J.size // max(nv, 1)
        r = _lib.CsRequest()
        r.nv, r.m = nv, m
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a.size else None
        r.M, r.J, r.qfrc, r.aref, r.D, r.g = p(M), p(J), p(q), p(ar), p(D), p(g)
        t = ctypes.c_uint64(0)
        _lib.check(self._lib.cs_serve_submit(self._h, ctypes.byref(r), ctypes.byref(t)),
                   "cs_serve_submit")
        self._shapes[t.value] = (nv, m)
        return int(t.value)

    def poll(self, ticket: int, outputs=True):
        """None while pending, else a dict with status, iters, times and (if
        ``outputs``) a, dqfrc, daref, dJ."""
        if ticket not in self._shapes:
            raise RuntimeError(f"unknown or retired ticket {ticket}")
        nv, m = self._shapes[ticket]
        res = _lib.CsResult()
        bufs = None
        if outputs:
            bufs = dict(a=np.empty(nv, np.float32), dqfrc=np.empty(nv, np.float32),
                        daref=np.empty(m, np.float32), dJ=np.empty((m, nv), np.float32))
            res.a = bufs["a"].ctypes.data
            res.dqfrc = bufs["dqfrc"].ctypes.data
            res.daref = bufs["daref"].ctypes.data if m else None
            res.dJ = bufs["dJ"].ctypes.data if m else None
        rc = self._lib.cs_serve_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(res))
        if rc == _lib.CS_PENDING:
            return None
        _lib.check(rc, "cs_serve_poll")
        del self._shapes[ticket]
        out = dict(status=res.status, iters=res.iters, t_submit=res.t_submit,
                   t_start=res.t_start, t_done=res.t_done)
        if bufs:
            out.update(bufs)
        return out

    # ---- bulk interface (one C call for many requests)
    @staticmethod
    def make_requests(items):
        """A ctypes array of cs_request for items (dicts with M, J, qfrc, aref,
        D, g float32 arrays); the arrays must stay alive while it is used."""
        arr = (_lib.CsRequest * len(items))()
        for i, p in enumerate(items):
            r = arr[i]
            nv = p["M"].shape[0]
            r.nv = nv
            r.m = p["J"].size // max(nv, 1)
            for k in ("M", "J", "qfrc", "aref", "D", "g"):
                a = p[k]
                setattr(r, k, a.ctypes.data if a.size else None)
        return arr

    def submit_batch(self, reqs, start, stop, tickets):
        """Queue reqs[start:stop] (a make_requests array); tickets is a
        ctypes uint64 array receiving their tickets at the same indices."""
        n = stop - start
        if n <= 0:
            return 0
        base = ctypes.cast(ctypes.byref(reqs, start * ctypes.sizeof(_lib.CsRequest)),
                           ctypes.POINTER(_lib.CsRequest))
        tk = ctypes.cast(ctypes.byref(tickets, start * 8), ctypes.POINTER(ctypes.c_uint64))
        rc = self._lib.cs_serve_submit_batch(self._h, n, base, tk)
        if rc < 0:
            _lib.check(rc, "cs_serve_submit_batch")
        return rc

    def clock(self) -> float:
        """The server's clock in seconds (cs_serve_clock)."""
        return float(self._lib.cs_serve_clock())

    def replay(self, reqs, t_arrival, t0, tickets) -> int:
        """Submit reqs (a make_requests array) at t0 + t_arrival[i] on the
        server's clock from native code (cs_serve_replay; the interpreter's
        lock is released for the call, so another thread can collect
        meanwhile); tickets (ctypes uint64 array) receives the tickets.
        Returns the number queued."""
        t = np.ascontiguousarray(t_arrival, dtype=np.float64)
        n = len(t)
        base = ctypes.cast(reqs, ctypes.POINTER(_lib.CsRequest))
        tp = t.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        tk = ctypes.cast(tickets, ctypes.POINTER(ctypes.c_uint64))
        rc = self._lib.cs_serve_replay(self._h, n, base, tp, float(t0), tk)
        if rc < 0:
            _lib.check(rc, "cs_serve_replay")
        return rc

    def poll_batch(self, tickets, start, stop, results, done):
        """Poll tickets[start:stop] without copying outputs; results (CsResult
        array) and done (int32 array) are filled at the same indices."""
        n = stop - start
        if n <= 0:
            return 0
        tk = ctypes.cast(ctypes.byref(tickets, start * 8), ctypes.POINTER(ctypes.c_uint64))
        rs = ctypes.cast(ctypes.byref(results, start * ctypes.sizeof(_lib.CsResult)),
                         ctypes.POINTER(_lib.CsResult))
        dn = ctypes.cast(ctypes.byref(done, start * 4), ctypes.POINTER(ctypes.c_int32))
        rc = self._lib.cs_serve_poll_batch(self._h, n, tk, rs, dn)
        return _lib.check(rc, "cs_serve_poll_batch")

    def completed(self, buf, max_n=None) -> int:
        """Tickets completed since the previous call (cs_serve_completed),
        written to buf (a ctypes uint64 array); returns their number."""
        n = len(buf) if max_n is None else int(max_n)
        rc = self._lib.cs_serve_completed(self._h, n, buf)
        return _lib.check(rc, "cs_serve_completed")

    def cancel(self, ticket: int):
        _lib.check(self._lib.cs_serve_cancel(self._h, ctypes.c_uint64(ticket)), "cs_serve_cancel")
        self._shapes.pop(ticket, None)

    def flush(self):
        _lib.check(self._lib.cs_serve_flush(self._h), "cs_serve_flush")

    def set_fault_hook(self, fn):
        """Host-side fault injection (cs_serve_set_fault_hook): fn(stage,
        batch) -> bool, True making that step of that batch fail; None
        removes it."""
        if fn is None:
            self._hook = None
            cb = _lib.SERVE_FAULT_FN()
        else:
            cb = _lib.SERVE_FAULT_FN(lambda stage, batch, user: 1 if fn(stage, batch) else 0)
            self._hook = cb   # the callback must outlive its use by the scheduler
        _lib.check(self._lib.cs_serve_set_fault_hook(self._h, cb, None),
                   "cs_serve_set_fault_hook")

    def stats(self) -> dict:
        s = _lib.CsServeStats()
        _lib.check(self._lib.cs_serve_get_stats(self._h, ctypes.byref(s)), "cs_serve_get_stats")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.cs_serve_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
