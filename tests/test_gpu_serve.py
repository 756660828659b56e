"""Serving (continuous batching): every result is the same alone and in the
mix, requests admitted while other batches are on the GPU overlap with them,
admission is bounded by device memory, and the fixed-batch baseline works."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2607_24959_b300 import serve, workloads as W
from tests import parity

pytestmark = pytest.mark.gpu


def _requests(n=120, seed=61):
    t, nv, nc = W.serve_stream(n_requests=n, seed=seed)
    return [W.serve_request(i, int(nv[i]), int(nc[i]), seed=seed) for i in range(n)]


def _wait(srv, tickets, timeout=60.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout, "serving timed out"
        time.sleep(1e-4)
    return [out[t] for t in tickets]


def _submit(srv, p):
    return srv.submit(p["M"], p["J"], p["qfrc"], p["aref"], p["D"], p["g"])


def test_alone_equals_mix_and_matches_oracle(cuda_device):
    reqs = _requests()
    with serve.Server(arena_bytes=256 << 20, streams=4) as srv:
        alone = [_wait(srv, [_submit(srv, p)])[0] for p in reqs]
        mixed = _wait(srv, [_submit(srv, p) for p in reqs])
        st = srv.stats()
    assert st["failed_launches"] == 0
    for p, a, b in zip(reqs, alone, mixed):
        assert a["status"] == b["status"] == 0
        for k in ("a", "dqfrc", "daref", "dJ"):
            assert np.array_equal(a[k], b[k]), k
    # parity of the served results against the oracle
    w = W.pack(reqs, name="served")
    ref = oracle.solve_workload(w, threads=8)
    gpu = dict(a=np.zeros(w.qfrc.size, np.float32), dqfrc=np.zeros(w.qfrc.size, np.float32),
               daref=np.zeros(w.aref.size, np.float32), dJ=np.zeros(w.J.size, np.float32),
               status=np.zeros(w.n, np.int32), iters=np.zeros(w.n, np.int32))
    for b, r in enumerate(mixed):
        e = w.inst[b]
        nv, m = int(e["nv"]), int(e["m"])
        gpu["a"][e["off_v"]:e["off_v"] + nv] = r["a"]
        gpu["dqfrc"][e["off_v"]:e["off_v"] + nv] = r["dqfrc"]
        gpu["daref"][e["off_r"]:e["off_r"] + m] = r["daref"]
        gpu["dJ"][e["off_J"]:e["off_J"] + m * nv] = r["dJ"].ravel()
        gpu["status"][b] = r["status"]
        gpu["iters"][b] = r["iters"]
    res = parity.compare(w, gpu, ref, np.arange(w.n))
    assert not res["bad"], res["bad"][:3]
    assert res["flipped"] <= 0.02 * w.n


def test_requests_admitted_while_others_run(cuda_device):
    reqs = _requests(n=400, seed=62)
    with serve.Server(arena_bytes=64 << 20, streams=4, max_batch=32) as srv:
        tickets = []

        def producer():
            for p in reqs:
                tickets.append(_submit(srv, p))
                time.sleep(2e-5)

        th = threading.Thread(target=producer)
        th.start()
        th.join()
        res = _wait(srv, list(tickets))
        st = srv.stats()
    assert all(r["status"] == 0 for r in res)
    assert st["batches"] >= 400 // 32
    assert st["max_inflight"] >= 2, st          # batches overlapped on the device
    starts = sorted(r["t_start"] for r in res)
    dones = sorted(r["t_done"] for r in res)
    assert starts[-1] > dones[0]                 # later requests started after earlier finished


def test_admission_by_device_memory(cuda_device):
    big = [W.serve_request(i, 96, 64, seed=63) for i in range(24)]   # ~150 KB each
    with serve.Server(arena_bytes=2 << 20, streams=2, max_batch=1000) as srv:
        res = _wait(srv, [_submit(srv, p) for p in big])
        st = srv.stats()
    assert all(r["status"] == 0 for r in res)
    # a 1 MiB slot holds at most ~6 of these requests, so the 24 need >= 4 batches
    assert st["batches"] >= 4, st


def test_fixed_policy_flush_and_cancel(cuda_device):
    reqs = _requests(n=70, seed=64)
    with serve.Server(arena_bytes=128 << 20, streams=1, policy="fixed", fixed_batch=32) as srv:
        ts = [_submit(srv, p) for p in reqs]
        time.sleep(0.5)
        st = srv.stats()
        assert st["batches"] == 2 and st["queued"] == 6, st
        srv.cancel(ts[-1])
        with pytest.raises(RuntimeError):
            srv.poll(ts[-1])
        srv.flush()
        res = _wait(srv, ts[:-1])
    assert all(r["status"] == 0 for r in res)


def test_bulk_submit_and_poll_out_of_order(cuda_device):
    import ctypes
    from paper_2607_24959_b300 import _lib
    reqs = _requests(n=200, seed=65)
    with serve.Server(arena_bytes=128 << 20, streams=4) as srv:
        carr = serve.Server.make_requests(reqs)
        tickets = (ctypes.c_uint64 * len(reqs))()
        results = (_lib.CsResult * len(reqs))()
        done = (ctypes.c_int32 * len(reqs))()
        assert srv.submit_batch(carr, 0, len(reqs), tickets) == len(reqs)
        t0 = time.time()
        while sum(done[i] == 1 for i in range(len(reqs))) < len(reqs):
            srv.poll_batch(tickets, 0, len(reqs), results, done)   # re-polls are skipped
            assert all(done[i] >= 0 for i in range(len(reqs)))
            assert time.time() - t0 < 60
            time.sleep(1e-3)
    assert all(results[i].status == 0 for i in range(len(reqs)))


def test_host_injected_launch_failure_on_the_gpu_server(cuda_device):
    """The fault hook on the CUDA server: batch 1's kernel launch is made to
    fail on the host (nothing is issued to the GPU for it); exactly its
    requests complete with CS_ST_FAILED, and the batches before and after it
    are solved as usual."""
    from paper_2607_24959_b300 import _lib
    reqs = _requests(n=12, seed=71)
    with serve.Server(arena_bytes=256 << 20, streams=2, policy="fixed",
                      fixed_batch=4) as srv:
        srv.set_fault_hook(lambda stage, batch: stage == _lib.SERVE_FAULT_LAUNCH and batch == 1)
        res = []
        for w in range(3):
            res += _wait(srv, [_submit(srv, p) for p in reqs[4 * w:4 * w + 4]])
        st = srv.stats()
        srv.set_fault_hook(None)
    assert [r["status"] for r in res] == [0] * 4 + [_lib.ST_FAILED] * 4 + [0] * 4
    assert all(not np.any(r["a"]) for r in res[4:8])
    assert st["failed_launches"] == 1 and st["batches"] == 3


def test_failure_after_some_bucket_kernels_were_launched(cuda_device):
    """A batch's four bucket kernels run on the slot's stream and its three
    auxiliary streams.  The third launch of batch 1 is made to fail on the
    host after the first two were issued: exactly that batch completes with
    CS_ST_FAILED, the slot is waited for on all of its streams and reused at
    once (one slot), and the next batch on it gives the results the same
    requests give alone."""
    from paper_2607_24959_b300 import _lib
    sizes = [(3, 2), (9, 10), (18, 20), (18, 40)]   # four (nv, rows) buckets
    reqs = [W.serve_request(100 + 4 * w + k, nv, nc, seed=72)
            for w in range(3) for k, (nv, nc) in enumerate(sizes)]
    calls = []

    def hook(stage, batch):
        if stage == _lib.SERVE_FAULT_LAUNCH and batch == 1:
            calls.append(1)
            return len(calls) == 3
        return False

    with serve.Server(arena_bytes=256 << 20, streams=1, policy="fixed",
                      fixed_batch=4) as srv:
        srv.set_fault_hook(hook)
        res = []
        for w in range(3):
            res += _wait(srv, [_submit(srv, p) for p in reqs[4 * w:4 * w + 4]])
        st = srv.stats()
        srv.set_fault_hook(None)
    assert len(calls) == 3
    assert [r["status"] for r in res] == [0] * 4 + [_lib.ST_FAILED] * 4 + [0] * 4
    assert st["failed_launches"] == 1 and st["batches"] == 3
    with serve.Server(arena_bytes=256 << 20, streams=1) as srv:
        alone = [_wait(srv, [_submit(srv, p)])[0] for p in reqs[8:]]
    for a, b in zip(alone, res[8:]):
        for k in ("a", "dqfrc", "daref", "dJ"):
            assert np.array_equal(a[k], b[k]), k
