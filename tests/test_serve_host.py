"""Serving failure handling and queue timeouts, on the host: the library's
scheduler (cs_serve_core.h) on a test double of the device
(tests/serve_host/fake_device.cpp), with failures injected through the fault
hook of the C ABI.  No GPU is used or faulted.

A batch whose input copy, kernel launch, output copy or completion fails
completes exactly its own requests with CS_ST_FAILED (outputs zeroed),
counts one failed launch, and leaves its slot free for the next batch;
requests that wait in the queue past queue_timeout_ms complete with
CS_ST_TIMEOUT without being run."""
import ctypes
import os
import subprocess
import time

import numpy as np
import pytest

from paper_2607_24959_b300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fake(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("serve_host") / "libfake_serve.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-pthread",
                           "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_2607_24959_b300", "csrc"),
                           os.path.join(ROOT, "tests", "serve_host", "fake_device.cpp"),
                           "-o", out])
    lib = ctypes.CDLL(out)
    vp = ctypes.c_void_p
    lib.fake_serve_create.argtypes = [ctypes.POINTER(_lib.CsServeConfig), ctypes.c_int,
                                      ctypes.POINTER(vp)]
    lib.fake_serve_submit.argtypes = [vp, ctypes.POINTER(_lib.CsRequest),
                                      ctypes.POINTER(ctypes.c_uint64)]
    lib.fake_serve_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(_lib.CsResult)]
    lib.fake_serve_flush.argtypes = [vp]
    lib.fake_serve_get_stats.argtypes = [vp, ctypes.POINTER(_lib.CsServeStats)]
    lib.fake_serve_set_fault_hook.argtypes = [vp, _lib.SERVE_FAULT_FN, vp]
    lib.fake_serve_replay.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(_lib.CsRequest),
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                      ctypes.POINTER(ctypes.c_uint64)]
    lib.fake_serve_clock.restype = ctypes.c_double
    lib.fake_serve_destroy.argtypes = [vp]
    lib.fake_serve_destroy.restype = None
    lib.fake_last_error.restype = ctypes.c_char_p
    return lib


class FakeServer:
    def __init__(self, lib, policy="fixed", fixed_batch=4, streams=2, latency_us=200,
                 queue_timeout_ms=0):
        self.lib = lib
        c = _lib.CsServeConfig()
        c.arena_bytes = streams * (8 << 20)
        c.streams = streams
        c.max_batch = 4096
        c.policy = _lib.CS_SERVE_FIXED if policy == "fixed" else _lib.CS_SERVE_CONTINUOUS
        c.fixed_batch = fixed_batch
        c.tol, c.max_iter, c.max_queue = 1e-8, 50, 0
        c.queue_timeout_ms = queue_timeout_ms
        self.h = ctypes.c_void_p()
        assert lib.fake_serve_create(ctypes.byref(c), latency_us, ctypes.byref(self.h)) == 0, \
            lib.fake_last_error()
        self.req = {}
        self._hook = None

    def submit(self, rng, nv=6, m=8):
        d = dict(M=np.eye(nv, dtype=np.float32), J=rng.standard_normal((m, nv)).astype(np.float32),
                 qfrc=rng.standard_normal(nv).astype(np.float32),
                 aref=rng.standard_normal(m).astype(np.float32),
                 D=np.full(m, 10.0, np.float32), g=rng.standard_normal(nv).astype(np.float32))
        r = _lib.CsRequest()
        r.nv, r.m = nv, m
        r.M, r.J, r.qfrc, r.aref, r.D, r.g = (d[k].ctypes.data for k in
                                              ("M", "J", "qfrc", "aref", "D", "g"))
        t = ctypes.c_uint64()
        assert self.lib.fake_serve_submit(self.h, ctypes.byref(r), ctypes.byref(t)) == 0
        self.req[t.value] = d
        return t.value

    def wait(self, tickets, timeout=5.0):
        out = {}
        t_end = time.monotonic() + timeout
        while len(out) < len(tickets):
            for t in tickets:
                if t in out:
                    continue
                nv, m = self.req[t]["qfrc"].size, self.req[t]["aref"].size
                bufs = dict(a=np.full(nv, 7.0, np.float32), dqfrc=np.full(nv, 7.0, np.float32),
                            daref=np.full(m, 7.0, np.float32),
                            dJ=np.full(m * nv, 7.0, np.float32))
                res = _lib.CsResult()
                res.a, res.dqfrc = bufs["a"].ctypes.data, bufs["dqfrc"].ctypes.data
                res.daref, res.dJ = bufs["daref"].ctypes.data, bufs["dJ"].ctypes.data
                rc = self.lib.fake_serve_poll(self.h, t, ctypes.byref(res))
                if rc == _lib.CS_PENDING:
                    continue
                assert rc == 0, self.lib.fake_last_error()
                out[t] = dict(status=res.status, iters=res.iters, t_submit=res.t_submit, **bufs)
            assert time.monotonic() < t_end, "requests did not complete"
            time.sleep(1e-3)
        return out

    def stats(self):
        s = _lib.CsServeStats()
        assert self.lib.fake_serve_get_stats(self.h, ctypes.byref(s)) == 0
        return {k: getattr(s, k) for k, _ in s._fields_}

    def set_hook(self, fn):
        self._hook = (_lib.SERVE_FAULT_FN(lambda st, b, u: 1 if fn(st, b) else 0)
                      if fn else _lib.SERVE_FAULT_FN())
        assert self.lib.fake_serve_set_fault_hook(self.h, self._hook, None) == 0

    def close(self):
        self.lib.fake_serve_destroy(self.h)


def _ok(srv, res):
    for t, r in res.items():
        d = srv.req[t]
        assert r["status"] == _lib.ST_OK and r["iters"] == 1
        assert np.array_equal(r["a"], d["qfrc"]) and np.array_equal(r["dqfrc"], d["g"])


def _failed(res, status):
    for r in res.values():
        assert r["status"] == status and r["iters"] == 0
        for k in ("a", "dqfrc", "daref", "dJ"):
            assert not np.any(r[k]), k       # outputs zeroed, not left as they were


@pytest.mark.parametrize("stage", [_lib.SERVE_FAULT_H2D, _lib.SERVE_FAULT_LAUNCH,
                                   _lib.SERVE_FAULT_D2H, _lib.SERVE_FAULT_COMPLETE])
def test_injected_failure_fails_exactly_that_batch(fake, stage):
    rng = np.random.default_rng(stage)
    srv = FakeServer(fake, fixed_batch=4)
    calls = []

    def hook(st, batch):
        calls.append((st, batch))
        return st == stage and batch == 1

    srv.set_hook(hook)
    try:
        waves = []
        for w in range(3):                     # batch w = wave w (fixed batches of 4)
            tk = [srv.submit(rng) for _ in range(4)]
            waves.append(srv.wait(tk))
        _ok(srv, waves[0])
        _failed(waves[1], _lib.ST_FAILED)
        _ok(srv, waves[2])                      # the slot was freed and reused
        st = srv.stats()
        assert st["failed_launches"] == 1 and st["completed"] == 12 and st["batches"] == 3
        assert (stage, 1) in calls
        assert {b for _, b in calls} == {0, 1, 2}
    finally:
        srv.close()


def test_failure_after_some_bucket_launches(fake):
    """A batch's bucket kernels are forked over the slot's stream and its
    auxiliary streams; a launch that fails after two of the batch's four
    bucket launches were issued fails exactly that batch, and the slot is
    reused by the next one."""
    rng = np.random.default_rng(11)
    srv = FakeServer(fake, fixed_batch=4, streams=1)
    sizes = [(6, 8), (6, 300), (40, 8), (40, 300)]   # four buckets of the fake device
    calls = []

    def hook(st, batch):
        if st == _lib.SERVE_FAULT_LAUNCH and batch == 1:
            calls.append(batch)
            return len(calls) == 3
        return False

    srv.set_hook(hook)
    try:
        waves = []
        for w in range(3):
            tk = [srv.submit(rng, nv=nv, m=m) for nv, m in sizes]
            waves.append(srv.wait(tk))
        _ok(srv, waves[0])
        _failed(waves[1], _lib.ST_FAILED)
        _ok(srv, waves[2])
        st = srv.stats()
        assert len(calls) == 3
        assert st["failed_launches"] == 1 and st["batches"] == 3
    finally:
        srv.close()


def test_failure_while_another_batch_is_in_flight(fake):
    rng = np.random.default_rng(7)
    srv = FakeServer(fake, fixed_batch=4, streams=2, latency_us=30000)
    srv.set_hook(lambda st, b: st == _lib.SERVE_FAULT_LAUNCH and b == 1)
    try:
        a = [srv.submit(rng) for _ in range(4)]       # batch 0: 30 ms on the "device"
        time.sleep(0.005)
        b = [srv.submit(rng) for _ in range(4)]       # batch 1: fails at launch
        c = [srv.submit(rng) for _ in range(4)]       # batch 2: reuses batch 1's slot
        rb = srv.wait(b)
        _failed(rb, _lib.ST_FAILED)
        ra, rc = srv.wait(a), srv.wait(c)
        _ok(srv, ra)
        _ok(srv, rc)
        st = srv.stats()
        assert st["failed_launches"] == 1 and st["max_inflight"] == 2
    finally:
        srv.close()


def test_queue_timeout(fake):
    rng = np.random.default_rng(8)
    # fixed batches of 1000 never fill: queued requests time out
    srv = FakeServer(fake, fixed_batch=1000, queue_timeout_ms=30)
    try:
        tk = [srv.submit(rng) for _ in range(5)]
        res = srv.wait(tk)
        _failed(res, _lib.ST_TIMEOUT)
        st = srv.stats()
        assert st["timed_out"] == 5 and st["batches"] == 0 and st["queued"] == 0
    finally:
        srv.close()
    # requests admitted before their deadline are not touched by it
    srv = FakeServer(fake, policy="continuous", queue_timeout_ms=1000)
    try:
        tk = [srv.submit(rng) for _ in range(16)]
        _ok(srv, srv.wait(tk))
        assert srv.stats()["timed_out"] == 0
    finally:
        srv.close()


def test_hook_removed(fake):
    rng = np.random.default_rng(9)
    srv = FakeServer(fake, fixed_batch=2)
    srv.set_hook(lambda st, b: True)
    try:
        _failed(srv.wait([srv.submit(rng) for _ in range(2)]), _lib.ST_FAILED)
        srv.set_hook(None)
        _ok(srv, srv.wait([srv.submit(rng) for _ in range(2)]))
    finally:
        srv.close()


def test_replay_submits_on_schedule(fake):
    """The native load generator (cs_serve_replay's core): every request is
    queued no earlier than its scheduled arrival on the server's clock and,
    on an idle host, shortly after it; all complete."""
    rng = np.random.default_rng(12)
    srv = FakeServer(fake, policy="continuous", streams=2, latency_us=100)
    try:
        n = 64
        data = [dict(M=np.eye(6, dtype=np.float32),
                     J=rng.standard_normal((8, 6)).astype(np.float32),
                     qfrc=rng.standard_normal(6).astype(np.float32),
                     aref=rng.standard_normal(8).astype(np.float32),
                     D=np.full(8, 10.0, np.float32),
                     g=rng.standard_normal(6).astype(np.float32)) for _ in range(n)]
        reqs = (_lib.CsRequest * n)()
        for r, d in zip(reqs, data):
            r.nv, r.m = 6, 8
            r.M, r.J, r.qfrc, r.aref, r.D, r.g = (d[k].ctypes.data for k in
                                                  ("M", "J", "qfrc", "aref", "D", "g"))
        t_arr = np.cumsum(rng.exponential(2e-4, n))          # about 5 k req/s
        tickets = (ctypes.c_uint64 * n)()
        t0 = fake.fake_serve_clock() + 0.01
        got = fake.fake_serve_replay(srv.h, n, reqs,
                                     t_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     t0, tickets)
        assert got == n
        for t, d in zip(tickets, data):
            srv.req[t] = d
        res = srv.wait(list(tickets))
        _ok(srv, res)
        lag = np.array([res[t]["t_submit"] for t in tickets]) - (t0 + t_arr)
        assert np.all(lag >= 0.0), lag.min()
        assert np.median(lag) < 5e-3, np.median(lag)
    finally:
        srv.close()
