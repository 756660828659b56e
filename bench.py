"""Benchmark: fused forward + IFT-adjoint contact solves per second.

Default workload: the quadruped horizon batch -- 512 trajectories x 64 steps =
32768 independent solves, nv = 18, contacts per instance uniform in 0..32
(4 pyramid rows each, so m in 0..128), FP32 on the GPU.  One step = one pass
of the whole hot path (stage, Newton solve with exact line search, IFT adjoint,
write a, dL/dqfrc, dL/daref, dL/dJ) over the batch, launched as one
CUDA-graph replay of the persistent fused kernel.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample instead (the reference arm of this benchmark).
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+IFT-adjoint contact solves/s at nv=18,nc=32; serve p50/p99 latency"
UNIT = "solves/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0, period_ms=20):
        self.index = index
        self.period_ms = period_ms
        self.proc = None
        self.lines = []   # (host monotonic time of arrival, csv line)
        self.marks = {}

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", f"-lms={self.period_ms}"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def wait_first(self, timeout=5.0):
        """Block until nvidia-smi has printed its first sample (or timeout)."""
        t_end = time.monotonic() + timeout
        while self.proc is not None and not self.lines and time.monotonic() < t_end:
            time.sleep(0.01)

    def mark(self, name):
        self.marks[name] = time.monotonic()

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, start=None, end=None):
        """Median SM clock, max clock and throttle reasons of the samples that
        arrived between marks `start` and `end` (all samples if unset)."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0 = self.marks.get(start, -1e300)
        t1 = self.marks.get(end, 1e300)
        for tt, ln in self.lines:
            if not (t0 <= tt <= t1):
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_work(inst, iters, act_counts):
    """Algorithmic FLOPs and bytes of one fused launch (per-instance sums).

    FLOPs: a0 = nv^3/3 + 2nv^2; per Newton iteration 4 m nv (J a, J^T f) +
    2 nv^2 (M a) + m_act nv (nv+1) (H) + nv^3/3 + 2 nv^2 (factor + solves) +
    2 m nv + 8 m (line search); the adjoint 2 nv^2 + 4 m nv; m_act is the
    final active count.  Bytes (4 B each): read M lower (nv(nv+1)/2), J (m nv),
    qfrc, g (2 nv), aref, D (2 m); write a, dqfrc (2 nv), daref (m), dJ (m nv).
    Work the algorithm does not need (padding, inactive rows in H, the
    compensated-arithmetic overhead, extra refinement passes) is not counted.
    """
    nv = inst["nv"].astype(np.float64)
    m = inst["m"].astype(np.float64)
    k = iters.astype(np.float64)
    ma = act_counts.astype(np.float64)
    per_it = 4 * m * nv + 2 * nv ** 2 + ma * nv * (nv + 1) + nv ** 3 / 3 + 2 * nv ** 2 \
        + 2 * m * nv + 8 * m
    flops = nv ** 3 / 3 + 2 * nv ** 2 + k * per_it + 2 * nv ** 2 + 4 * m * nv
    byts = 4 * (nv * (nv + 1) / 2 + m * nv + 2 * nv + 2 * m + 2 * nv + m + m * nv)
    return float(flops.sum()), float(byts.sum())


def elliptic_work(inst, iters, act_contacts):
    """Algorithmic FLOPs and bytes of one round-cone fused solve per instance
    (sums over the batch), k its Newton steps and c_act its contacts outside
    zone 0 at the returned point, m = 3 nc.  FLOPs: a0 = nv^3/3 + 2 nv^2; per
    step the residual 2 m nv (J a) + 2 nv^2 (M a) + 6 c_act nv (J^T grad) +
    40 nc (cone evaluation), the Newton matrix c_act (18 nv + 3 nv (nv+1))
    (hess J_c, then J_c^T of it, lower triangle), nv^3/3 + 2 nv^2 (factor and
    solves), and the line search 2 m nv + 2 nv^2 + 40 nc (one evaluation
    counted); the adjoint 2 nv^2 + 4 m nv, the gradients 2 m nv + 2 nv^2 +
    30 nc.  Bytes (4 B each): read M lower, J, qfrc, g, aref, D, mu; write a,
    dqfrc, daref, dD, dmu, dJ and dM."""
    nv = inst["nv"].astype(np.float64)
    m = inst["m"].astype(np.float64)
    nc = m / 3
    k = iters.astype(np.float64)
    ca = act_contacts.astype(np.float64)
    per_it = (2 * m * nv + 2 * nv ** 2 + 6 * ca * nv + 40 * nc
              + ca * (18 * nv + 3 * nv * (nv + 1)) + nv ** 3 / 3 + 2 * nv ** 2
              + 2 * m * nv + 2 * nv ** 2 + 40 * nc)
    flops = nv ** 3 / 3 + 2 * nv ** 2 + k * per_it + 2 * nv ** 2 + 4 * m * nv \
        + 2 * m * nv + 2 * nv ** 2 + 30 * nc
    byts = 4 * (nv * (nv + 1) / 2 + m * nv + 2 * nv + 3 * m
                + 2 * nv + 3 * m + m * nv + nv * nv)
    return float(flops.sum()), float(byts.sum())


def ncg_work(inst, iters, act_counts):
    """Algorithmic FLOPs of the conjugate-gradient forward plus the IFT
    adjoint per instance (sums over the batch), k its CG steps: a0 and the
    factor of M nv^3/3 + 2 nv^2; per step the residual 2 m nv + 2 m_act nv +
    2 nv^2, the M^-1 preconditioner 2 nv^2, the line search 2 m nv + 2 nv^2 +
    8 m; the adjoint's Newton matrix m_act nv (nv+1), its factor and solve
    nv^3/3 + 2 nv^2, and 2 nv^2 + 4 m nv.  Bytes as the Newton path's."""
    nv = inst["nv"].astype(np.float64)
    m = inst["m"].astype(np.float64)
    k = iters.astype(np.float64)
    ma = act_counts.astype(np.float64)
    per_it = 2 * m * nv + 2 * ma * nv + 2 * nv ** 2 + 2 * nv ** 2 + 2 * m * nv + 2 * nv ** 2 + 8 * m
    flops = (nv ** 3 / 3 + 2 * nv ** 2 + k * per_it + ma * nv * (nv + 1) + nv ** 3 / 3
             + 2 * nv ** 2 + 2 * nv ** 2 + 4 * m * nv)
    byts = 4 * (nv * (nv + 1) / 2 + m * nv + 2 * nv + 2 * m + 2 * nv + m + m * nv)
    return float(flops.sum()), float(byts.sum())


def roofline_obj(flops, byts, t_s, dev):
    """The roofline object of a leg: the larger of its FP32 and HBM
    fractions (measured peaks) names the bound."""
    import torch
    peaks, _ = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * 2 * float(peaks.get("sm_max_mhz", 2032.0)) * 1e6 / 1e12
    hbm_peak = float(peaks.get("hbm_gbs", 6400.0))
    frac_alu = flops / t_s / 1e12 / fp32_peak
    frac_hbm = byts / t_s / 1e9 / hbm_peak
    alu = frac_alu >= frac_hbm
    return {"bound": "alu" if alu else "hbm",
            "achieved": flops / t_s / 1e12 if alu else byts / t_s / 1e9,
            "peak": fp32_peak if alu else hbm_peak,
            "unit": "TFLOP/s" if alu else "GB/s", "frac": max(frac_alu, frac_hbm),
            "traffic": None, "hbm_frac": frac_hbm, "alu_frac": frac_alu,
            "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": byts}


# DRAM bytes (read + write) of one step of the fused warp kernels on the
# 32768-instance quadruped batch: ncu dram__bytes_read.sum +
# dram__bytes_write.sum of the four bucket kernels of the second of two
# consecutive plan replays, caches not flushed between kernels (so the write-
# backs of earlier outputs are counted where they happen).  Valid for the
# kernel sources whose hash is recorded; any change of them makes the figure
# stale and the bench line then reports traffic as null.
QUADRUPED_STEP_TRAFFIC = {
    "instances": 32768, "read": 242078720, "write": 167943232,
    "sources_sha1": "d75555e2d3c14655ecd2ca9adace685880da83bb",
    "how": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --cache-control none "
           "on the full quadruped batch, mean of replays 2-5 of the four bucket kernels"}


def kernel_sources_sha1():
    """Hash of the sources the quadruped step's kernels and launches are built
    from: the warp solver, its launcher and nv = 18 instantiation, and the
    plan (the CTA solver, serving and other paths do not run in that step;
    the public header holds declarations only)."""
    import hashlib
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2607_24959_b300", "csrc")
    files = [os.path.join(csrc, f) for f in ("cs_warp.cuh", "cs_launch.cuh", "cs_kern_nv18.cu",
                                             "cs_host.h", "cs_plan.cu")]
    for f in files:
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode())
            h.update(fh.read())
    return h.hexdigest()


def make_workload(name, rank, n=None):
    from paper_2607_24959_b300 import workloads as W
    seed_shift = 7919 * rank
    kw = {} if n is None else {"n": n}
    if name == "quadruped":
        return W.quadruped(seed=W.SEEDS["quadruped"] + seed_shift, **kw)
    if name == "franka":
        return W.franka(seed=W.SEEDS["franka"] + seed_shift, **kw)
    if name == "tiny":
        return W.tiny(seed=W.SEEDS["tiny"] + seed_shift, **kw)
    if name == "nv96":
        return W.nv96(seed=W.SEEDS["nv96"] + seed_shift, **kw)
    if name == "nc256":
        return W.nc256(seed=W.SEEDS["nc256"] + 1 + seed_shift, **kw)
    raise SystemExit(f"unknown workload {name}")


def workload_config(name, w):
    p = w.params
    return {"workload": f"{name}: {w.n} solves, nv={p['nv']}, m=4*nc, "
                        f"nc~U{{0..{w.m_max // 4}}}" if name == "quadruped" else
            f"{name}: {w.n} solves, nv={p['nv']}, m={w.m_max}",
            "instances": w.n, "nv": p["nv"], "m_max": w.m_max,
            "mean_m": float(w.inst["m"].mean()), "cond_M": p["cond"],
            "D_range": list(p["d_range"]), "seed": p["seed"]}


def cpu_baseline(w, max_instances=None, threads=None, single_sample=2048, repeats=5):
    """The FP64 oracle, as it stands, on the host cores: the whole sample on
    every core (threads claim chunks of 64 instances), and the first
    `single_sample` instances of it on one core.  Inputs are converted to the
    oracle's float64 arrays before the clock starts; one untimed pass, then
    the median of `repeats` timed passes (one pass is a fraction of a second,
    and the first one also pays for the output pages and the threads)."""
    import oracle
    threads = threads or (os.cpu_count() or 1)
    n = w.n if max_instances is None else min(w.n, max_instances)
    ws = w if n == w.n else w.subset(np.arange(n))
    oracle.build()

    def timed(pw, th):
        pw.run_all(threads=th)
        ts = []
        for _ in range(max(1, repeats)):
            t0 = time.perf_counter()
            pw.run_all(threads=th)
            ts.append(time.perf_counter() - t0)
        return statistics.median(ts)

    pw = oracle.PreparedWorkload(ws)
    dt = timed(pw, threads)
    res = {"value": n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"first {n} of the {w.n} instances, forward + adjoint, "
                     f"{threads} threads, median of {repeats} passes of {dt:.3f} s wall"}
    if single_sample:
        n1 = min(n, single_sample)
        w1 = ws if n1 == ws.n else ws.subset(np.arange(n1))
        d1 = timed(oracle.PreparedWorkload(w1), 1)
        res["single_thread"] = {"value": n1 / d1, "unit": UNIT, "cores": 1,
                                "sample": f"first {n1} instances, one thread, median of "
                                          f"{repeats} passes of {d1:.3f} s wall"}
    res["build"] = "gcc -O3 -march=native -std=c99 -ffp-contract=off"
    res["iters_mean"] = float(pw.iters.mean()) if n else 0.0
    return res


def _serve_pool(n_requests, rate, seed, pool_per_class=2048):
    """Arrival times and a pool of request data per nv class (requests of a
    class cycle through its pool; data drawn like the serving workload)."""
    from paper_2607_24959_b300 import workloads as W
    t, nv, nc = W.serve_stream(n_requests=n_requests, rate=rate, seed=seed)
    pools = {}
    for k, v in enumerate(sorted(set(nv.tolist()))):
        sel = np.flatnonzero(nv == v)
        P = int(min(pool_per_class, max(1, sel.size)))
        w = W.generate(f"serve-nv{v}", P, int(v), nc[sel[:P]], seed=seed * 7 + k,
                       cond=1e4 if v >= 96 else 1e3)
        pools[int(v)] = [{kk: np.ascontiguousarray(x) for kk, x in w.instance(b).items()}
                         for b in range(P)]
    reqs = []
    counters = {v: 0 for v in pools}
    for i in range(n_requests):
        v = int(nv[i])
        reqs.append(pools[v][counters[v] % len(pools[v])])
        counters[v] += 1
    return t, reqs


def serve_run(t_arr, reqs, policy, fixed_batch=1024, streams=8, arena_bytes=2 << 30,
              clients=1):
    """Replay the arrivals against a server (cs_serve_replay submits them on
    schedule from native code; this thread collects through the bulk C
    calls); latency = completion - scheduled arrival on the server's clock
    (so any lag of the client counts too)."""
    import ctypes
    from paper_2607_24959_b300 import _lib, serve
    from paper_2607_24959_b300 import workloads as W
    n = len(reqs)
    srv = serve.Server(arena_bytes=arena_bytes, streams=streams if policy != "fixed" else 1,
                       max_batch=8192, policy=policy, fixed_batch=fixed_batch)
    # warm-up before the stream, as a deployed server would: one request per
    # (nv, rows-per-lane) kernel variant, so that no first-use module load of
    # a kernel falls inside the measured stream, and 512 requests of the
    # stream's mix, so that the server's buffer pool is populated
    warm = [W.serve_request(10**9 + i, nv, nc) for i, (nv, nc) in enumerate(
        (nv, nc) for nv in (3, 9, 18, 96) for nc in (0, 8, 16, 24, 32, 48, 64))]
    warm += reqs[:512]   # and the buffer pool holds a stream's worth of buffers
    wt = [srv.submit(r["M"], r["J"], r["qfrc"], r["aref"], r["D"], r["g"]) for r in warm]
    if policy == "fixed":
        srv.flush()
    for tk in wt:
        while srv.poll(tk) is None:
            time.sleep(1e-4)
    drain = (ctypes.c_uint64 * 8192)()
    while srv.completed(drain):      # the warm-up's completions are not the stream's
        pass
    # the stream's tickets follow the warm-up's without a gap, in submission
    # order (they are global to the server, whichever thread submits)
    base_ticket = max(int(tk) for tk in wt) + 1
    subsets = [np.arange(j, n, clients) for j in range(clients)]
    carrs = [serve.Server.make_requests([reqs[i] for i in sub]) for sub in subsets]
    tks = [(ctypes.c_uint64 * len(sub))() for sub in subsets]
    t0 = srv.clock() + 0.05
    submitted = [0] * clients

    def producer(j):
        # the arrivals are submitted on schedule from native code
        # (cs_serve_replay), so the client's own lag does not depend on the
        # interpreter; the thread releases the interpreter's lock meanwhile.
        # With several clients each replays every clients-th arrival.
        submitted[j] = srv.replay(carrs[j], t_arr[subsets[j]], t0, tks[j])

    def producers():
        ths = [threading.Thread(target=producer, args=(j,), daemon=True) for j in range(clients)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        if policy == "fixed":
            srv.flush()

    th = threading.Thread(target=producers, daemon=True)
    th.start()
    # collect exactly the tickets the server reports as completed (no scan
    # of the outstanding ones under the server's lock)
    t_done = np.zeros(n)
    t_sub = np.zeros(n)
    t_start = np.zeros(n)
    status = np.full(n, -1, np.int64)
    comp = (ctypes.c_uint64 * 8192)()
    rtmp = (_lib.CsResult * 8192)()
    dtmp = (ctypes.c_int32 * 8192)()
    collected = 0
    deadline = time.monotonic() + 120.0 + float(t_arr[-1])
    while collected < n:
        k = srv.completed(comp)
        if k:
            for i in range(k):
                dtmp[i] = 0
            srv.poll_batch(comp, 0, k, rtmp, dtmp)
            for i in range(k):
                if dtmp[i] != 1:
                    srv.close()
                    raise RuntimeError("serving lost a ticket")
                idx = int(comp[i]) - base_ticket      # submission position
                t_done[idx] = rtmp[i].t_done
                t_sub[idx] = rtmp[i].t_submit
                t_start[idx] = rtmp[i].t_start
                status[idx] = rtmp[i].status
            collected += k
        else:
            time.sleep(1e-4)
        if time.monotonic() > deadline:
            srv.close()
            raise RuntimeError(f"serving did not finish: {collected} of {n} collected")
    th.join(timeout=10.0)
    st = srv.stats()
    srv.close()
    # from submission positions back to the stream's order
    perm = np.empty(n, np.int64)
    for sub, tk in zip(subsets, tks):
        perm[np.frombuffer(tk, dtype=np.uint64).astype(np.int64) - base_ticket] = sub
    for arr in (t_done, t_sub, t_start, status):
        arr[perm] = arr.copy()
    lat = t_done - (t0 + np.asarray(t_arr))
    span = t_done.max() - (t0 + t_arr[0])
    # where the latency goes: the client's lag behind the scheduled arrival,
    # the wait in the server's queue, and the batch's GPU round trip
    # (staging, copies, kernels, completion), medians and 99th percentiles
    parts = {"client_lag": t_sub - (t0 + np.asarray(t_arr)), "queue": t_start - t_sub,
             "service": t_done - t_start}
    split = {k: {"p50_ms": float(np.percentile(v, 50) * 1e3),
                 "p99_ms": float(np.percentile(v, 99) * 1e3)} for k, v in parts.items()}
    nvs = np.array([len(r["qfrc"]) for r in reqs])
    split["by_nv"] = {int(v): {"p50_ms": float(np.percentile(lat[nvs == v], 50) * 1e3),
                               "p99_ms": float(np.percentile(lat[nvs == v], 99) * 1e3),
                               "queue_p50_ms": float(np.percentile(parts["queue"][nvs == v], 50) * 1e3),
                               "service_p50_ms": float(np.percentile(parts["service"][nvs == v], 50) * 1e3)}
                      for v in np.unique(nvs)}
    return {"requests": n, "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "latency_split": split,
            "mean_ms": float(lat.mean() * 1e3), "solves_per_s": n / span,
            "ok": int(np.sum(status == 0)),
            "status_counts": {int(k): int(v) for k, v in zip(*np.unique(status, return_counts=True))},
            "batches": int(st["batches"]),
            "mean_batch": st["batched_requests"] / max(st["batches"], 1),
            "max_inflight": int(st["max_inflight"])}


def run_serve(args):
    """Serving stream (Poisson arrivals, nv in {3,9,18,96}, nc in 0..64):
    continuous batching next to fixed-size launches of the same requests; then
    a sweep of the arrival rate (the same mix, fewer requests per rate above
    the headline one) to find where each policy stops keeping up."""
    t_arr, reqs = _serve_pool(args.serve_requests, args.serve_rate, 1005)
    cont = serve_run(t_arr, reqs, "continuous", streams=args.serve_streams,
                     clients=args.serve_clients)
    fixed = serve_run(t_arr, reqs, "fixed", fixed_batch=args.serve_fixed_batch,
                      clients=args.serve_clients)
    out = {"requests": args.serve_requests, "rate_per_s": args.serve_rate,
           "mix": "nv {3,9,18,96} p {.3,.3,.3,.1}, nc U{0..64}, fwd + adjoint each",
           "client_threads": args.serve_clients,
           "continuous": cont, f"fixed_{args.serve_fixed_batch}": fixed}
    sweep = []
    for rate in [float(r) for r in args.serve_sweep.split(",") if r]:
        n = int(min(args.serve_requests, max(20000, rate * 0.4)))
        t_s, r_s = _serve_pool(n, rate, 1005)
        row = {"rate_per_s": rate, "requests": n}
        for pol in ("continuous", "fixed"):
            res = serve_run(t_s, r_s, pol, fixed_batch=args.serve_fixed_batch,
                            streams=args.serve_streams, clients=args.serve_clients)
            row[pol] = {k: res[k] for k in ("p50_ms", "p99_ms", "solves_per_s", "ok",
                                            "mean_batch", "max_inflight")}
            row[pol]["latency_split"] = {k: res["latency_split"][k]
                                         for k in ("client_lag", "queue", "service")}
        sweep.append(row)
    if sweep:
        out["rate_sweep"] = sweep
        out["rate_sweep_note"] = ("each row is its own stream of Poisson arrivals at that rate; "
                                  "a policy keeps up while solves_per_s matches the rate, and its "
                                  "latency grows without bound past that knee")
    return out


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, each step one
    cpu_baseline() pass over the same instances the GPU arm's cpu_baseline
    leg times (the whole workload by default)."""
    ws_, rank = _dist()
    if rank != 0:
        return
    w = make_workload(args.workload, 0, args.n)
    n_sample = min(w.n, args.cpu_sample)
    for _ in range(args.warmup):
        cpu_baseline(w, max_instances=min(256, n_sample), single_sample=0, repeats=1)
    vals = [cpu_baseline(w, max_instances=n_sample, single_sample=0, repeats=1)
            for _ in range(args.steps)]
    v = statistics.median([x["value"] for x in vals])
    one = cpu_baseline(w, max_instances=n_sample)["single_thread"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * n_sample / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(args.workload, w),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"],
                             "kind": "oracle", "sample": vals[0]["sample"]
                             + f"; median of {args.steps} steps",
                             "single_thread": one, "build": vals[0]["build"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bench_config(name, w):
    """The `config` object both arms print for a workload."""
    return dict(workload_config(name, w),
                l2="inputs+outputs 330 MB per step exceed the 126 MB L2; no flush",
                graph="one CUDA-graph replay per step (plan)",
                claim_order="per bucket, cost-descending, dynamic counter",
                precision="FP32 with compensated residuals and refinement: a returned "
                          "when the untaken Newton correction, or the error a refinement "
                          "step leaves (predicted from consecutive corrections), is <= "
                          "1e-7 max|a| (one FP32 ulp), the adjoint refined to 1e-5 |w| / "
                          "3e-5 |lambda| the same way; parity 1e-4 (a) / 1e-3 (gradients) "
                          "relative to an FP64 oracle (measured worst 7e-7 / 3.4e-5); the "
                          "paper's experiments use FP64")


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2607_24959_b300 import solver, _lib

    world, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _lib.load()
    w = make_workload(args.workload, rank, args.n)
    batch = solver.DeviceBatch.from_workload(w, dev)
    g = torch.from_numpy(w.g).to(dev)
    order = torch.from_numpy(solver.cost_order(w.inst)).to(dev)
    out = solver.alloc_fused(batch)
    kw = dict(order=order, tol=args.tol, max_iter=args.max_iter,
              warps_per_block=args.warps_per_block)

    # plan: per-(nv, m) bucket kernels, cost-ordered claims, autotuned
    # warps per block, captured as one CUDA graph (tuning runs happen here)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        plan = solver.FusedPlan(batch, g, tol=args.tol, max_iter=args.max_iter,
                                autotune=args.warps_per_block == 0, graph=True,
                                warps_per_block=args.warps_per_block, out=out)
    torch.cuda.synchronize()
    plan_info = plan.describe()
    # clocks are sampled from before the warm-up to the end of the timed
    # region; the warm-up runs at least W steps and at least 0.5 s so that
    # samples under this same load exist even when K steps take milliseconds
    clk = ClockSampler(index=local).__enter__()
    clk.wait_first()
    clk.mark("warmup")
    t_w = time.monotonic()
    with torch.cuda.stream(stream):
        n_w = 0
        while n_w < args.warmup or time.monotonic() - t_w < args.warmup_seconds:
            plan.launch()
            n_w += 1
            if n_w % 16 == 0:
                stream.synchronize()
    torch.cuda.synchronize()

    # ---- timed region: K graph replays on `stream`
    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    clk.mark("timed")
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(args.steps):
            plan.launch()
        ev1.record(stream)
    barrier()
    clk.mark("end")
    time.sleep(0.05)   # the sample in flight at the end of the timed region
    clk.__exit__(None, None, None)
    ms_total = ev0.elapsed_time(ev1)
    t = torch.tensor([ms_total], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_total = float(t.item())
    ms_step = ms_total / args.steps
    total_solves = w.n * world * args.steps
    value = total_solves / (ms_total / 1e3)

    status = out.status.cpu().numpy()[:w.n]
    iters = out.iters.cpu().numpy()[:w.n]
    daref = out.daref.cpu().numpy()
    act_counts = np.array([np.count_nonzero(daref[o:o + mm]) for o, mm in
                           zip(w.inst["off_r"], w.inst["m"])])
    flops, byts = algorithmic_work(w.inst, iters, act_counts)
    peaks, peak_src = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * 2 * float(peaks.get("sm_max_mhz", 2032.0)) * 1e6 / 1e12  # TFLOP/s
    hbm_peak = float(peaks.get("hbm_gbs", 6400.0))
    t_s = ms_step / 1e3
    tflops = flops / t_s / 1e12
    gbs = byts / t_s / 1e9
    frac_alu = tflops / fp32_peak
    frac_hbm = gbs / hbm_peak
    if frac_alu >= frac_hbm:
        roof = {"bound": "alu", "achieved": tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": frac_alu, "traffic": None,
                "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 x "
                               f"{peaks.get('sm_max_mhz', 2032.0)} MHz ({peak_src} clock)",
                "hbm": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                        "frac": frac_hbm, "peak_source": f"{peak_src} hbm_gbs"}}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": frac_hbm, "traffic": None}
    if args.workload == "quadruped" and w.n == QUADRUPED_STEP_TRAFFIC["instances"]:
        if kernel_sources_sha1() == QUADRUPED_STEP_TRAFFIC["sources_sha1"]:
            roof["traffic"] = QUADRUPED_STEP_TRAFFIC["read"] + QUADRUPED_STEP_TRAFFIC["write"]
            roof["traffic_read"] = QUADRUPED_STEP_TRAFFIC["read"]
            roof["traffic_write"] = QUADRUPED_STEP_TRAFFIC["write"]
            roof["traffic_source"] = QUADRUPED_STEP_TRAFFIC["how"]
        else:
            roof["traffic_source"] = "null: the kernel sources changed since the ncu capture"
    roof["kernel"] = "warp_solve_kernel<NV,MT,FUSED> buckets (all launches of one step)"
    roof["algorithmic_flops_per_launch"] = flops
    roof["algorithmic_bytes_per_launch"] = byts

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, w, batch, dev, kw, world)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": bench_config(args.workload, w),
            "roofline": roof,
            "clocks": dict(clk.summary("warmup", "end"),
                           window="nvidia-smi samples from the start of the warm-up "
                                  f"({n_w} replays, >= {args.warmup_seconds} s) to the end "
                                  "of the timed region",
                           timed_region=clk.summary("timed", "end")),
            "gpu_launches": args.steps * plan_info["kernels"], "plan": plan_info,
            "status_counts": np.bincount(status, minlength=6).tolist(),
            "iters_mean": float(iters.mean()), "iters_max": int(iters.max())}
    if e2e:
        line["e2e"] = e2e
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(w, max_instances=args.cpu_sample)
        line["oracle_iters_mean"] = line["cpu_baseline"].pop("iters_mean", None)
    if args.configs and world == 1:
        line["configs"] = run_configs(args, peaks, peak_src)
    if not args.no_serve and world == 1:
        del plan, out, batch
        torch.cuda.empty_cache()
        line["serve"] = run_serve(args)
    if not args.no_memory and world == 1:
        line["adjoint_memory"] = run_memory(args)
    if not args.no_elliptic and world == 1:
        line["elliptic"] = run_elliptic(args)
    if not args.no_ncg and world == 1:
        line["ncg"] = run_ncg(args)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_configs(args, peaks, peak_src):
    """The other configurations of the benchmark suite, each on its own: the
    fused forward + adjoint through a plan (bucketed, autotuned, one CUDA
    graph), CUDA-event timed on the plan's stream after warm-up, with the same
    roofline accounting and an oracle baseline on the host cores."""
    import torch
    from paper_2607_24959_b300 import solver

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * 2 * float(peaks.get("sm_max_mhz", 2032.0)) * 1e6 / 1e12
    hbm_peak = float(peaks.get("hbm_gbs", 6400.0))
    legs = {}
    for name in args.configs.split(","):
        if not name:
            continue
        w = make_workload(name, 0)
        batch = solver.DeviceBatch.from_workload(w, dev)
        g = torch.from_numpy(w.g).to(dev)
        out = solver.alloc_fused(batch)
        stream = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(stream):
            plan = solver.FusedPlan(batch, g, tol=args.tol, max_iter=args.max_iter,
                                    autotune=True, graph=True, out=out)
            t_w = time.monotonic()
            n_w = 0
            while n_w < 3 or time.monotonic() - t_w < 0.2:
                plan.launch()
                n_w += 1
            steps = max(5, min(args.steps, 100))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                plan.launch()
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        st = out.status.cpu().numpy()[:w.n]
        it = out.iters.cpu().numpy()[:w.n]
        daref = out.daref.cpu().numpy()
        act = np.array([np.count_nonzero(daref[o:o + mm]) for o, mm in
                        zip(w.inst["off_r"], w.inst["m"])])
        flops, byts = algorithmic_work(w.inst, it, act)
        t_s = ms / 1e3
        frac_alu = flops / t_s / 1e12 / fp32_peak
        frac_hbm = byts / t_s / 1e9 / hbm_peak
        info = plan.describe()
        plan.close()
        legs[name] = {
            "metric": "fwd+IFT-adjoint contact solves/s", "value": w.n / t_s, "unit": UNIT,
            "ms_per_step": ms, "steps": steps, "config": workload_config(name, w),
            "roofline": {"bound": "alu" if frac_alu >= frac_hbm else "hbm",
                         "achieved": flops / t_s / 1e12 if frac_alu >= frac_hbm
                         else byts / t_s / 1e9,
                         "peak": fp32_peak if frac_alu >= frac_hbm else hbm_peak,
                         "unit": "TFLOP/s" if frac_alu >= frac_hbm else "GB/s",
                         "frac": max(frac_alu, frac_hbm), "traffic": None,
                         "hbm_frac": frac_hbm, "alu_frac": frac_alu,
                         "algorithmic_flops_per_launch": flops,
                         "algorithmic_bytes_per_launch": byts},
            "plan": info, "status_counts": np.bincount(st, minlength=6).tolist(),
            "iters_mean": float(it.mean()), "iters_max": int(it.max()),
            "gpu_launches_per_step": info["kernels"]}
        if not args.no_cpu_baseline:
            cb = cpu_baseline(w, repeats=3)
            legs[name]["cpu_baseline"] = cb
        del out, batch, g
        torch.cuda.empty_cache()
    return legs


def run_memory(args):
    """The paper's memory comparison (Section III-E, Fig. 3), on B300 with
    this library's kernels: device bytes for differentiating the solve with
    the IFT adjoint (state independent of K) against unrolled reverse mode
    (trace grows with K), through the autograd wrappers, B = 1024 instances.
    The three sweeps of the figure's panels: step cap K = 1..10 at nv 24 with
    4 contacts; contacts 1..256 at nv 6, K = 5; N particles (nv 6N, N
    contacts) for N = 1..16, K = 5.  Instances up to nv 32 and 256 rows run
    one warp each, larger ones one CTA each (both paths).  The paper's two
    headline ratios (256 contacts at nv 6; 16 particles, nv 96) are printed
    beside ours."""
    import torch
    from paper_2607_24959_b300 import autograd as csag, solver, workloads as W

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))

    def measure(w, K, methods=("ift", "unrolled")):
        batch = solver.DeviceBatch.from_workload(w, dev)
        g = torch.from_numpy(w.g).to(dev)
        res = {}
        for name in methods:
            def once():
                J = batch.J.clone().requires_grad_(True)
                q = batch.qfrc.clone().requires_grad_(True)
                if name == "ift":
                    a = csag.contact_solve(batch, J=J, qfrc=q, max_iter=K)
                else:
                    a = csag.contact_solve_unrolled(batch, J=J, qfrc=q, K=K)
                (a[:g.numel()] * g).sum().backward()
                return J, q
            once()
            times = []
            for rep in range(3):
                # autograd graphs of earlier calls are freed before the peak
                # is taken, and the collector does not run inside it
                torch.cuda.synchronize()
                gc.collect()
                gc.disable()
                try:
                    torch.cuda.reset_peak_memory_stats(dev)
                    base = torch.cuda.memory_allocated(dev)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    J, q = once()
                    e1.record()
                    torch.cuda.synchronize()
                    peak = torch.cuda.max_memory_allocated(dev) - base
                finally:
                    gc.enable()
                times.append(e0.elapsed_time(e1))
                del J, q
            if name == "ift":
                kept = solver.alloc_state(batch, True).nbytes()
            else:
                kept = solver.unrolled_fwd(batch, K).nbytes()
            res[name] = {"kept_bytes": int(kept), "peak_bytes": int(peak),
                         "ms": round(float(np.median(times)), 4)}
        del batch, g
        torch.cuda.empty_cache()
        return res

    out = {"method": "bytes kept between forward and backward (IFT: a_lo, active set, "
                     "factor of H(a*); unrolled: per-step factor, a_k, p_k, alpha_k, c1_k, "
                     "masks) and peak device bytes allocated during one forward + backward "
                     "through the autograd wrappers (torch allocator, inputs excluded), FP32; "
                     "J and qfrc require grad",
           "batch": 1024}
    ks = list(range(1, 11))
    w = W.generate("mem-iter", 1024, 24, 4, seed=71, cond=1e2)
    rows = [measure(w, K) for K in ks]
    out["iterations"] = {
        "config": "nv 24, 4 contacts (16 rows), cond(M) 1e2, B 1024", "K": ks,
        "ift_peak": [r["ift"]["peak_bytes"] for r in rows],
        "unrolled_peak": [r["unrolled"]["peak_bytes"] for r in rows],
        "ift_kept": [r["ift"]["kept_bytes"] for r in rows],
        "unrolled_kept": [r["unrolled"]["kept_bytes"] for r in rows],
        "ift_ms": [r["ift"]["ms"] for r in rows],
        "unrolled_ms": [r["unrolled"]["ms"] for r in rows]}
    it = out["iterations"]
    it["ift_peak_change_K1_to_K10"] = it["ift_peak"][-1] / it["ift_peak"][0] - 1.0
    it["unrolled_peak_growth_K1_to_K10"] = it["unrolled_peak"][-1] / it["unrolled_peak"][0]
    ncs = [1, 2, 4, 8, 16, 32, 64, 128, 256]
    rows = [measure(W.generate(f"mem-c{nc}", 1024, 6, nc, seed=72 + nc, cond=1e2), 5)
            for nc in ncs]
    out["contacts"] = {
        "config": "nv 6, K 5, B 1024", "contacts": ncs,
        "ift_peak": [r["ift"]["peak_bytes"] for r in rows],
        "unrolled_peak": [r["unrolled"]["peak_bytes"] for r in rows],
        "unrolled_over_ift": [r["unrolled"]["peak_bytes"] / r["ift"]["peak_bytes"]
                              for r in rows]}
    Ns = [1, 2, 3, 4, 6, 8, 12, 16]
    rows = [measure(W.generate(f"mem-n{N}", 1024, 6 * N, N, seed=80 + N, cond=1e2), 5)
            for N in Ns]
    out["dof"] = {
        "config": "N particles: nv 6N, N contacts, K 5, B 1024", "N": Ns,
        "ift_peak": [r["ift"]["peak_bytes"] for r in rows],
        "unrolled_peak": [r["unrolled"]["peak_bytes"] for r in rows],
        "unrolled_over_ift": [r["unrolled"]["peak_bytes"] / r["ift"]["peak_bytes"]
                              for r in rows]}
    c, d = out["contacts"], out["dof"]
    out["headline"] = {
        "contacts_256_nv6": {"ift_peak": c["ift_peak"][-1], "unrolled_peak": c["unrolled_peak"][-1],
                             "unrolled_over_ift": c["unrolled_over_ift"][-1], "paper": 20.0},
        "particles_16_nv96": {"ift_peak": d["ift_peak"][-1], "unrolled_peak": d["unrolled_peak"][-1],
                              "unrolled_over_ift": d["unrolled_over_ift"][-1], "paper": 6.0},
        "paper_setting": "compiled temporary memory of JAX/XLA MJX programs, FP64, B 1024, K 5, "
                         "on a 4 GiB GPU (paper, Fig. 3); here FP32 device bytes of this "
                         "library's kernels on one B300"}
    # the scaling extremes run one CTA per instance, beyond the unrolled
    # path's one-warp sizes: the IFT adjoint's memory against the step cap
    ext = {"config": "IFT adjoint through the autograd wrapper, step cap K; nv96: nv 96, "
                     "16 contacts (64 rows), cond(M) 1e4, B 2048; nc256: nv 18, 256 contacts "
                     "(1024 rows), B 256", "K": ks}
    for label, w in (("nv96", W.nv96(seed=W.SEEDS["nv96"])),
                     ("nc256", W.nc256(seed=W.SEEDS["nc256"] + 1))):
        rows = [measure(w, K, ("ift",)) for K in ks]
        peaks = [r["ift"]["peak_bytes"] for r in rows]
        ext[label] = {"ift_peak": peaks, "ift_kept": [r["ift"]["kept_bytes"] for r in rows],
                      "ift_ms": [r["ift"]["ms"] for r in rows],
                      "ift_peak_change_K1_to_K10": peaks[-1] / peaks[0] - 1.0}
    out["scaling_extremes"] = ext
    return out


def run_elliptic(args):
    """The same workload shape with MuJoCo's round cone (three rows per
    contact, Eqs. 2-5): one fused launch of cs_solve_fused_elliptic per step
    over the 32768-instance batch (one warp per instance), cost-ordered
    claims, CUDA-event timed on its stream after warm-up; and the paper's
    16-particle size (nv 96, 16 round-cone contacts, one CTA per instance,
    2048 instances) the same way."""
    import torch
    from paper_2607_24959_b300 import solver, workloads as W

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))

    def timed(w, max_steps):
        batch = solver.DeviceBatch.from_workload(w, dev)
        g = torch.from_numpy(w.g).to(dev)
        mu = torch.from_numpy(w.mu).to(dev)
        order = torch.from_numpy(solver.cost_order(w.inst)).to(dev)
        out = solver.solve_fused_elliptic(batch, g, mu, order=order, tol=args.tol)
        stream = torch.cuda.Stream(device=dev)
        steps = max(3, min(args.steps, max_steps))
        with torch.cuda.stream(stream):
            for _ in range(max(args.warmup, 3)):
                solver.solve_fused_elliptic(batch, g, mu, order=order, tol=args.tol, out=out)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                solver.solve_fused_elliptic(batch, g, mu, order=order, tol=args.tol, out=out)
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        st = out.fused.status.cpu().numpy()[:w.n]
        it = out.fused.iters.cpu().numpy()[:w.n]
        daref = out.fused.daref.cpu().numpy()
        # contacts outside zone 0 at the returned point: nonzero lambda rows
        ca = np.array([np.count_nonzero(np.abs(daref[o:o + mm]).reshape(-1, 3).sum(1))
                       if mm else 0 for o, mm in zip(w.inst["off_r"], w.inst["m"])])
        flops, byts = elliptic_work(w.inst, it, ca)
        roof = roofline_obj(flops, byts, ms / 1e3, dev)
        del out, batch
        torch.cuda.empty_cache()
        return ms, steps, st, it, roof

    w = W.quadruped_elliptic(n=args.elliptic_n)
    ms, steps, st, it, roof = timed(w, 50)
    res = {"metric": "round-cone fwd+IFT-adjoint solves/s (all parameter gradients)",
           "value": w.n / (ms / 1e3), "unit": "solves/s", "ms_per_step": ms, "steps": steps,
           "config": {"workload": "quadruped_elliptic", "instances": w.n, "nv": 18,
                      "contacts": "U{0..32}, 3 rows each", "mu": "U(0.2, 1.2)"},
           "status_counts": np.bincount(st, minlength=6).tolist(),
           "iters_mean": float(it.mean()), "iters_max": int(it.max()),
           "gpu_launches_per_step": 1, "roofline": roof}
    w = W.generate("nv96_elliptic", 2048, 96, 16, seed=97, cond=1e3, cone="elliptic")
    ms, steps, st, it, roof = timed(w, 20)
    res["nv96"] = {"value": w.n / (ms / 1e3), "unit": "solves/s", "ms_per_step": ms,
                   "steps": steps,
                   "config": {"workload": "nv96_elliptic", "instances": w.n, "nv": 96,
                              "contacts": 16, "rows": 48, "cond_M": 1e3,
                              "kernel": "one CTA per instance"},
                   "status_counts": np.bincount(st, minlength=6).tolist(),
                   "iters_mean": float(it.mean()), "iters_max": int(it.max()),
                   "gpu_launches_per_step": 1, "roofline": roof}
    return res


def run_ncg(args):
    """The headline batch solved by nonlinear conjugate gradients (the other
    forward solver of Section III-B) feeding the same IFT adjoint: one fused
    launch per step, CUDA-event timed."""
    import torch
    from paper_2607_24959_b300 import solver, workloads as W

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    w = W.quadruped()
    batch = solver.DeviceBatch.from_workload(w, dev)
    g = torch.from_numpy(w.g).to(dev)
    order = torch.from_numpy(solver.cost_order(w.inst)).to(dev)
    out = solver.solve_fused_ncg(batch, g, order=order, tol=args.tol)
    stream = torch.cuda.Stream(device=dev)
    steps = 3
    with torch.cuda.stream(stream):
        solver.solve_fused_ncg(batch, g, order=order, tol=args.tol, out=out)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            solver.solve_fused_ncg(batch, g, order=order, tol=args.tol, out=out)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    st = out.status.cpu().numpy()[:w.n]
    it = out.iters.cpu().numpy()[:w.n]
    daref = out.daref.cpu().numpy()
    act = np.array([np.count_nonzero(daref[o:o + mm]) for o, mm in
                    zip(w.inst["off_r"], w.inst["m"])])
    flops, byts = ncg_work(w.inst, it, act)
    res = {"metric": "fwd+IFT-adjoint solves/s with the conjugate-gradient forward solver",
           "value": w.n / (ms / 1e3), "unit": "solves/s", "ms_per_step": ms, "steps": steps,
           "config": {"workload": "quadruped", "instances": w.n,
                      "max_iter": solver.NCG_MAX_ITER},
           "status_counts": np.bincount(st, minlength=6).tolist(),
           "iters_mean": float(it.mean()), "iters_max": int(it.max()),
           "roofline": roofline_obj(flops, byts, ms / 1e3, dev)}
    del out, batch
    torch.cuda.empty_cache()
    return res


def run_e2e(args, w, batch, dev, kw, world):
    """Same metric through the public API with pinned host buffers: every step
    copies its inputs host->device and its results device->host
    (solver.HostPipeline: chunked, copies overlapped with the solves)."""
    import torch
    from paper_2607_24959_b300 import solver

    pipe = solver.HostPipeline(w, chunks=args.e2e_chunks, device=dev, tol=args.tol,
                               max_iter=args.max_iter)
    h2d, d2h = pipe.bytes_per_step()
    for _ in range(max(args.warmup, 1)):
        pipe.step()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 50))
    t0 = time.perf_counter()
    for _ in range(steps):
        pipe.step()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    st = pipe.h_out["status"].numpy()[:w.n]
    pipe.close()
    return {"value": w.n * world * steps / (ms / 1e3), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": ms / steps, "steps": steps, "chunks": len(pipe.chunks),
            "status_ok": int(np.sum(st == 0)),
            "timing": "host wall clock over the steps, synchronised at both ends"}


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="quadruped")
    ap.add_argument("--n", type=int, default=None,
                    help="instances (default: the workload's full size)")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--max-iter", type=int, default=50)
    ap.add_argument("--warps-per-block", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=32768)
    ap.add_argument("--configs", default="tiny,franka,nv96,nc256",
                    help="comma-separated workloads measured beside the headline one "
                         "(empty to skip)")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-ncg", action="store_true",
                    help="skip the conjugate-gradient forward solver leg")
    ap.add_argument("--no-elliptic", action="store_true",
                    help="skip the round-cone throughput leg")
    ap.add_argument("--elliptic-n", type=int, default=32768,
                    help="instances of the round-cone leg's quadruped batch")
    ap.add_argument("--no-memory", action="store_true",
                    help="skip the IFT vs unrolled differentiation memory sweeps")
    ap.add_argument("--warmup-seconds", type=float, default=0.5,
                    help="warm-up replays continue for at least this long (clock samples "
                         "under load); 0 leaves exactly --warmup replays, as a profiler "
                         "capture of the timed launches wants")
    ap.add_argument("--e2e-chunks", type=int, default=4)
    ap.add_argument("--serve-requests", type=int, default=200000)
    ap.add_argument("--serve-rate", type=float, default=50000.0)
    ap.add_argument("--serve-fixed-batch", type=int, default=1024)
    ap.add_argument("--serve-streams", type=int, default=8,
                    help="batches in flight at once for the continuous policy (1..16)")
    ap.add_argument("--serve-clients", type=int, default=1,
                    help="client threads replaying the arrivals (each every n-th one)")
    ap.add_argument("--serve-sweep", default="200000,500000,1000000",
                    help="arrival rates (req/s) of the serving sweep; empty to skip")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
