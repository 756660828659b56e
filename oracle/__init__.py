"""FP64 CPU oracle for the batched smooth-contact solve and its IFT adjoint.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` are the only callers.  The product
path (``paper_2607_24959_b300``) never imports this package.

The arithmetic lives in ``cs_oracle.c`` (plain C, double precision); this
module compiles it with gcc on first use and marshals numpy arrays through
ctypes.  Every function follows the paper's Section III:

* ``solve_one``    Newton on the stationarity residual (Eqs. 6, 8, 9, 10) with
                   an exact line search and exact termination.
* ``adjoint_one``  the transposed solve of Eq. 17 at the returned point.
* ``adjoint_theta_one`` the same, adding the M and D terms of Eq. 17.
* ``ell_*``       the same solve and adjoint with MuJoCo's round Coulomb
                   cone (three rows per contact, Eqs. 2-5) instead of the
                   pyramid rows.
* ``unrolled_one`` / ``unrolled_workload``  the derivative through the
                   executed trace of at most K Newton steps (the unrolled
                   reverse-mode sensitivity the paper compares with IFT).
* ``residual_one`` / ``objective_one``  Eq. 8 and Eq. 5 evaluated at a point.
* ``solve_workload`` the same over a packed ragged batch, optionally on
                   several host threads (each thread runs the unchanged
                   single-instance code on its own slice of instances).

Parity pins (closed forms, brute-force active sets in exact rational
arithmetic, central differences, an independently written unrolled-Newton
derivative) are in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cs_oracle.c")
_lock = threading.Lock()
_lib = None

STATUS = {0: "OK", 1: "MAXITER", 2: "CHOLFAIL", 3: "NONFINITE", 4: "BADSHAPE",
          5: "NOPROGRESS"}
DEFAULT_TOL = 1e-12
DEFAULT_MAX_ITER = 100


def _host_signature() -> str:
    """A short key of this host's CPU (model and instruction-set flags): the
    library is compiled with -march=native, so a copy built on another machine
    must not be loaded here."""
    import hashlib
    key = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith(("model name", "flags", "Features", "CPU part")):
                    key += line
                    if line.startswith(("flags", "Features")):
                        break
    except OSError:
        pass
    return hashlib.sha1(key.encode()).hexdigest()[:12]


def lib_path() -> str:
    return os.path.join(_HERE, f"_cs_oracle-{_host_signature()}.so")


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O3 -march=native, ISO C99: no FMA contraction
    and no fast-math, so every result is the plain double-precision
    evaluation of the source) if it is missing or stale for this host."""
    lib = lib_path()
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= os.path.getmtime(_SRC)):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O3", "-march=native", "-std=c99",
                           "-ffp-contract=off", "-fPIC", "-shared", _SRC,
                           "-o", tmp, "-lm"])
    os.replace(tmp, lib)
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            ip = ctypes.POINTER(ctypes.c_int)
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            ci, cd = ctypes.c_int, ctypes.c_double
            lib.oracle_solve.argtypes = [ci, ci, dp, dp, dp, dp, dp, dp, cd, ci,
                                         dp, u8p, ip]
            lib.oracle_solve.restype = ci
            lib.oracle_adjoint.argtypes = [ci, ci, dp, dp, dp, dp, dp, dp, dp,
                                           dp, dp, dp, u8p]
            lib.oracle_adjoint.restype = ci
            lib.oracle_residual.argtypes = [ci, ci, dp, dp, dp, dp, dp, dp, dp,
                                            dp, u8p]
            lib.oracle_residual.restype = cd
            lib.oracle_objective.argtypes = [ci, ci, dp, dp, dp, dp, dp, dp]
            lib.oracle_objective.restype = cd
            lib.oracle_batch.argtypes = [ci, ci, i32p, i32p, i64p, i64p, i64p,
                                         i64p, dp, dp, dp, dp, dp, dp, cd, ci,
                                         dp, u8p, i32p, i32p, dp, dp, dp, dp,
                                         dp]
            lib.oracle_batch.restype = None
            lib.oracle_adjoint_theta.argtypes = [ci, ci, dp, dp, dp, dp, dp, dp,
                                                 dp, dp, dp, dp, dp, dp, u8p]
            lib.oracle_adjoint_theta.restype = ci
            lib.oracle_unrolled.argtypes = [ci, ci, dp, dp, dp, dp, dp, dp, ci,
                                            cd, dp, ip, dp, dp, dp, dp, dp]
            lib.oracle_unrolled.restype = ci
            lib.oracle_ell_cone.argtypes = [dp, cd, cd, cd, dp, dp, dp]
            lib.oracle_ell_cone.restype = ci
            lib.oracle_ell_solve.argtypes = [ci, ci, dp, dp, dp, dp, dp, dp, cd, ci,
                                             dp, u8p, ip]
            lib.oracle_ell_solve.restype = ci
            lib.oracle_ell_adjoint.argtypes = [ci, ci, dp, dp, dp, dp, dp, dp, dp, dp,
                                               dp, dp, dp, dp, dp, dp, u8p]
            lib.oracle_ell_adjoint.restype = ci
            lib.oracle_ell_objective.argtypes = [ci, ci, dp, dp, dp, dp, dp, dp, dp]
            lib.oracle_ell_objective.restype = cd
            lib.oracle_ell_line_search.argtypes = [ci, ci, dp, dp, dp, dp, dp, dp, dp,
                                                   dp]
            lib.oracle_ell_line_search.restype = cd
            lib.oracle_line_search.argtypes = [ci, ci, dp, dp, dp, dp, dp, dp,
                                               dp]
            lib.oracle_line_search.restype = cd
            _lib = lib
    return _lib


def _d(x):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    return x, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _prob(M, J, qfrc, aref, D):
    M = np.asarray(M, np.float64)
    nv = M.shape[0]
    J = np.asarray(J, np.float64).reshape(-1, nv)
    return nv, J.shape[0], [_d(M), _d(J), _d(qfrc), _d(aref), _d(D)]


def solve_one(M, J, qfrc, aref, D, a_init=None, tol=DEFAULT_TOL,
              max_iter=DEFAULT_MAX_ITER):
    """Returns (a, act, status, iters) for one instance."""
    lib = _load()
    nv, m, arrs = _prob(M, J, qfrc, aref, D)
    a = np.zeros(nv)
    act = np.zeros(max(m, 1), np.uint8)
    it = ctypes.c_int(0)
    ai = None if a_init is None else _d(a_init)
    st = lib.oracle_solve(nv, m, *[p for _, p in arrs],
                          None if ai is None else ai[1], tol, max_iter,
                          a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          act.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                          ctypes.byref(it))
    return a, act[:m].astype(bool), int(st), int(it.value)


def adjoint_one(M, J, qfrc, aref, D, a, g):
    """Returns (dqfrc, daref, dJ, act, status) of Eq. 17 at the point a."""
    lib = _load()
    nv, m, arrs = _prob(M, J, qfrc, aref, D)
    _, ap = _d(a)
    _, gp = _d(g)
    aa = _d(a)[0]
    dq = np.zeros(nv)
    dr = np.zeros(max(m, 1))
    dJ = np.zeros(max(m * nv, 1))
    act = np.zeros(max(m, 1), np.uint8)
    c = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = lib.oracle_adjoint(nv, m, *[p for _, p in arrs], c(aa), gp, c(dq),
                            c(dr), c(dJ),
                            act.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return dq, dr[:m], dJ[:m * nv].reshape(m, nv), act[:m].astype(bool), int(st)


def adjoint_theta_one(M, J, qfrc, aref, D, a, g):
    """Returns (dqfrc, daref, dJ, dM, dD, act, status): Eq. 17 for every
    parameter, dM being the derivative with respect to a symmetric M."""
    lib = _load()
    nv, m, arrs = _prob(M, J, qfrc, aref, D)
    aa = _d(a)[0]
    gp = _d(g)[1]
    dq = np.zeros(nv)
    dr = np.zeros(max(m, 1))
    dJ = np.zeros(max(m * nv, 1))
    dM = np.zeros(nv * nv)
    dD = np.zeros(max(m, 1))
    act = np.zeros(max(m, 1), np.uint8)
    c = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = lib.oracle_adjoint_theta(
        nv, m, *[p for _, p in arrs], c(aa), gp, c(dq), c(dr), c(dJ), c(dM),
        c(dD), act.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return (dq, dr[:m], dJ[:m * nv].reshape(m, nv), dM.reshape(nv, nv), dD[:m],
            act[:m].astype(bool), int(st))


def unrolled_one(M, J, qfrc, aref, D, g, K, tol=DEFAULT_TOL):
    """Derivative of g^T a_K through the executed trace of at most K Newton
    steps (unrolled reverse mode, Section III-E).  Returns a dict with a (the
    returned a_K), steps, status and dqfrc, daref, dJ, dM (symmetric M), dD."""
    lib = _load()
    nv, m, arrs = _prob(M, J, qfrc, aref, D)
    gp = _d(g)[1]
    a = np.zeros(nv)
    dq = np.zeros(nv)
    dr = np.zeros(max(m, 1))
    dJ = np.zeros(max(m * nv, 1))
    dM = np.zeros(nv * nv)
    dD = np.zeros(max(m, 1))
    steps = ctypes.c_int(0)
    c = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = lib.oracle_unrolled(nv, m, *[p for _, p in arrs], gp, int(K), float(tol),
                             c(a), ctypes.byref(steps), c(dq), c(dr), c(dJ), c(dM),
                             c(dD))
    return dict(a=a, steps=int(steps.value), status=int(st), dqfrc=dq, daref=dr[:m],
                dJ=dJ[:m * nv].reshape(m, nv), dM=dM.reshape(nv, nv), dD=dD[:m])


def unrolled_workload(w, K, idx=None, tol=DEFAULT_TOL, threads=1):
    """unrolled_one over a packed ragged batch (with the workload's g).
    Returns packed float64 a, dqfrc, daref, dJ, dM, dD and per-instance
    status and steps; instances outside ``idx`` stay zero."""
    inst = w.inst
    n = inst.shape[0]
    out = dict(a=np.zeros(w.qfrc.size), dqfrc=np.zeros(w.qfrc.size),
               daref=np.zeros(w.aref.size), dJ=np.zeros(w.J.size),
               dM=np.zeros(w.M.size), dD=np.zeros(w.aref.size),
               status=np.full(n, -1, np.int32), iters=np.zeros(n, np.int32))
    todo = np.arange(n) if idx is None else np.asarray(idx).ravel()

    def run(bs):
        for b in bs:
            e = inst[int(b)]
            nv, m = int(e["nv"]), int(e["m"])
            ov, orr, oJ, oM = (int(e[k]) for k in ("off_v", "off_r", "off_J", "off_M"))
            p = w.instance(int(b))
            res = unrolled_one(p["M"], p["J"], p["qfrc"], p["aref"], p["D"], p["g"], K,
                               tol)
            out["a"][ov:ov + nv] = res["a"]
            out["dqfrc"][ov:ov + nv] = res["dqfrc"]
            out["daref"][orr:orr + m] = res["daref"]
            out["dD"][orr:orr + m] = res["dD"]
            out["dJ"][oJ:oJ + m * nv] = res["dJ"].ravel()
            out["dM"][oM:oM + nv * nv] = res["dM"].ravel()
            out["status"][int(b)] = res["status"]
            out["iters"][int(b)] = res["steps"]

    if threads <= 1 or todo.size < 2:
        run(todo)
    else:
        ts = [threading.Thread(target=run, args=(part,))
              for part in np.array_split(todo, threads) if part.size]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
    return out


# ---- round (elliptic) cone: three rows per contact (normal, two tangents),
# D_N = D[3c], D_T = D[3c+1] (D[3c+2] not read), mu = mu[3c].

def _c(x):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def ell_cone_one(u, DN, DT, mu):
    """(zone, s, grad[3], hess[3x3]) of one contact's round-cone cost."""
    lib = _load()
    uu = _d(u)[0]
    s = ctypes.c_double(0.0)
    g = np.zeros(3)
    h = np.zeros(9)
    z = lib.oracle_ell_cone(_c(uu), float(DN), float(DT), float(mu), ctypes.byref(s),
                            _c(g), _c(h))
    return int(z), float(s.value), g, h.reshape(3, 3)


def ell_solve_one(M, J, qfrc, aref, D, mu, tol=DEFAULT_TOL, max_iter=DEFAULT_MAX_ITER):
    """Returns (a, zone per row, status, iters) with the round cone."""
    lib = _load()
    nv, m, arrs = _prob(M, J, qfrc, aref, D)
    muu = _d(mu)[0]
    a = np.zeros(nv)
    zone = np.zeros(max(m, 1), np.uint8)
    it = ctypes.c_int(0)
    st = lib.oracle_ell_solve(nv, m, *[p for _, p in arrs], _c(muu), float(tol),
                              int(max_iter), _c(a),
                              zone.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                              ctypes.byref(it))
    return a, zone[:m].copy(), int(st), int(it.value)


def ell_adjoint_one(M, J, qfrc, aref, D, mu, a, g):
    """Eq. 17 with the round cone at a: dict of dqfrc, daref, dJ, dM, dD, dmu,
    zone, status."""
    lib = _load()
    nv, m, arrs = _prob(M, J, qfrc, aref, D)
    muu, aa, gg = _d(mu)[0], _d(a)[0], _d(g)[0]
    out = dict(dqfrc=np.zeros(nv), daref=np.zeros(max(m, 1)), dJ=np.zeros(max(m * nv, 1)),
               dM=np.zeros(nv * nv), dD=np.zeros(max(m, 1)), dmu=np.zeros(max(m, 1)))
    zone = np.zeros(max(m, 1), np.uint8)
    st = lib.oracle_ell_adjoint(nv, m, *[p for _, p in arrs], _c(muu), _c(aa), _c(gg),
                                *[_c(out[k]) for k in ("dqfrc", "daref", "dJ", "dM", "dD",
                                                       "dmu")],
                                zone.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    out["daref"] = out["daref"][:m]
    out["dD"] = out["dD"][:m]
    out["dmu"] = out["dmu"][:m]
    out["dJ"] = out["dJ"][:m * nv].reshape(m, nv)
    out["dM"] = out["dM"].reshape(nv, nv)
    out["zone"] = zone[:m].copy()
    out["status"] = int(st)
    return out


def ell_objective_one(M, J, qfrc, aref, D, mu, a):
    lib = _load()
    nv, m, arrs = _prob(M, J, qfrc, aref, D)
    return float(lib.oracle_ell_objective(nv, m, *[p for _, p in arrs], _c(_d(mu)[0]),
                                          _c(_d(a)[0])))


def ell_line_search_one(M, J, qfrc, aref, D, mu, a, p):
    lib = _load()
    nv, m, arrs = _prob(M, J, qfrc, aref, D)
    return float(lib.oracle_ell_line_search(nv, m, *[q for _, q in arrs], _c(_d(mu)[0]),
                                            _c(_d(a)[0]), _c(_d(p)[0])))


def ell_solve_workload(w, idx=None, tol=DEFAULT_TOL, max_iter=DEFAULT_MAX_ITER,
                       threads=1):
    """Round-cone forward + adjoint (with the workload's g and mu) over a
    packed batch: packed a, dqfrc, daref, dJ, dM, dD, dmu, zone and
    per-instance status and iters; instances outside ``idx`` stay zero."""
    inst = w.inst
    n = inst.shape[0]
    out = dict(a=np.zeros(w.qfrc.size), dqfrc=np.zeros(w.qfrc.size),
               daref=np.zeros(w.aref.size), dJ=np.zeros(w.J.size), dM=np.zeros(w.M.size),
               dD=np.zeros(w.aref.size), dmu=np.zeros(w.aref.size),
               zone=np.zeros(w.aref.size, np.uint8), status=np.full(n, -1, np.int32),
               iters=np.zeros(n, np.int32))
    todo = np.arange(n) if idx is None else np.asarray(idx).ravel()

    def run(bs):
        for b in bs:
            e = inst[int(b)]
            nv, m = int(e["nv"]), int(e["m"])
            ov, orr, oJ, oM = (int(e[k]) for k in ("off_v", "off_r", "off_J", "off_M"))
            p = w.instance(int(b))
            a, zone, st, it = ell_solve_one(p["M"], p["J"], p["qfrc"], p["aref"], p["D"],
                                            p["mu"], tol, max_iter)
            out["a"][ov:ov + nv] = a
            out["status"][int(b)] = st
            out["iters"][int(b)] = it
            out["zone"][orr:orr + m] = zone
            if st in (2, 3, 4):
                continue
            adj = ell_adjoint_one(p["M"], p["J"], p["qfrc"], p["aref"], p["D"], p["mu"], a,
                                  p["g"])
            if adj["status"]:
                out["status"][int(b)] = adj["status"]
            out["dqfrc"][ov:ov + nv] = adj["dqfrc"]
            out["daref"][orr:orr + m] = adj["daref"]
            out["dD"][orr:orr + m] = adj["dD"]
            out["dmu"][orr:orr + m] = adj["dmu"]
            out["dJ"][oJ:oJ + m * nv] = adj["dJ"].ravel()
            out["dM"][oM:oM + nv * nv] = adj["dM"].ravel()

    if threads <= 1 or todo.size < 2:
        run(todo)
    else:
        ts = [threading.Thread(target=run, args=(part,))
              for part in np.array_split(todo, threads) if part.size]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
    return out


def residual_one(M, J, qfrc, aref, D, a):
    """Returns (r, f, act, scale) of Eq. 8 at the point a."""
    lib = _load()
    nv, m, arrs = _prob(M, J, qfrc, aref, D)
    aa = _d(a)[0]
    r = np.zeros(nv)
    f = np.zeros(max(m, 1))
    act = np.zeros(max(m, 1), np.uint8)
    c = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    scale = lib.oracle_residual(nv, m, *[p for _, p in arrs], c(aa), c(r), c(f),
                                act.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return r, f[:m], act[:m].astype(bool), float(scale)


def objective_one(M, J, qfrc, aref, D, a):
    """The reduced objective of Eq. 5 at a (pyramidal rows)."""
    lib = _load()
    nv, m, arrs = _prob(M, J, qfrc, aref, D)
    aa = _d(a)[0]
    return float(lib.oracle_objective(
        nv, m, *[p for _, p in arrs],
        aa.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))


def line_search_one(M, J, qfrc, aref, D, a, p):
    """The exact step length argmin_{alpha>0} L(a + alpha p) (Eqs. 5, 10)."""
    lib = _load()
    nv, m, arrs = _prob(M, J, qfrc, aref, D)
    aa = _d(a)[0]
    pp = _d(p)[0]
    c = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return float(lib.oracle_line_search(nv, m, *[q for _, q in arrs], c(aa),
                                        c(pp)))


class PreparedWorkload:
    """A packed batch converted once to the oracle's float64 / int arrays,
    with its output arrays; ``run`` solves instances [lo, hi)."""

    def __init__(self, w, tol=DEFAULT_TOL, max_iter=DEFAULT_MAX_ITER, adjoint=True,
                 theta=False):
        self.lib = _load()
        inst = w.inst
        self.n = n = inst.shape[0]
        self.nv = np.ascontiguousarray(inst["nv"], np.int32)
        self.m = np.ascontiguousarray(inst["m"], np.int32)
        self.offs = [np.ascontiguousarray(inst[k], np.int64)
                     for k in ("off_M", "off_J", "off_v", "off_r")]
        self.M, self.J, self.q, self.ar, self.D, self.g = (
            np.ascontiguousarray(x, np.float64)
            for x in (w.M, w.J, w.qfrc, w.aref, w.D, w.g))
        self.tol, self.max_iter, self.adjoint, self.theta = tol, max_iter, adjoint, theta
        self.a = np.zeros(max(self.q.size, 1))
        self.dq = np.zeros(max(self.q.size, 1))
        self.dr = np.zeros(max(self.ar.size, 1))
        self.dJ = np.zeros(max(self.J.size, 1))
        self.act = np.zeros(max(self.ar.size, 1), np.uint8)
        self.dM = np.zeros(max(self.M.size, 1)) if theta else None
        self.dD = np.zeros(max(self.ar.size, 1)) if theta else None
        self.status = np.full(n, -1, np.int32)
        self.iters = np.zeros(n, np.int32)
        P = ctypes.POINTER
        cd = lambda x: None if x is None else x.ctypes.data_as(P(ctypes.c_double))
        ci32 = lambda x: x.ctypes.data_as(P(ctypes.c_int32))
        ci64 = lambda x: x.ctypes.data_as(P(ctypes.c_int64))
        # pointers taken once: a call of run() only crosses into the C code
        self._ptrs = ([ci32(self.nv), ci32(self.m)] + [ci64(o) for o in self.offs]
                      + [cd(self.M), cd(self.J), cd(self.q), cd(self.ar), cd(self.D),
                         cd(self.g) if adjoint else None])
        self._outs = [cd(self.a), self.act.ctypes.data_as(P(ctypes.c_uint8)),
                      ci32(self.status), ci32(self.iters), cd(self.dq), cd(self.dr),
                      cd(self.dJ), cd(self.dM), cd(self.dD)]

    def run(self, lo, hi):
        self.lib.oracle_batch(lo, hi, *self._ptrs, self.tol, self.max_iter, *self._outs)

    def run_all(self, threads=1, chunk=64):
        """Every instance, on `threads` host threads that claim chunks of
        `chunk` consecutive instances from a shared counter (ctypes releases
        the GIL during the C call, so the threads run in parallel)."""
        n = self.n
        if threads <= 1 or n <= chunk:
            if n:
                self.run(0, n)
            return
        lock = threading.Lock()
        nxt = [0]

        def worker():
            while True:
                with lock:
                    lo = nxt[0]
                    nxt[0] = lo + chunk
                if lo >= n:
                    return
                self.run(lo, min(n, lo + chunk))

        ts = [threading.Thread(target=worker) for _ in range(threads)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()

    def outputs(self):
        out = dict(a=self.a[:self.q.size], dqfrc=self.dq[:self.q.size],
                   daref=self.dr[:self.ar.size], dJ=self.dJ[:self.J.size],
                   act=self.act[:self.ar.size], status=self.status, iters=self.iters)
        if self.theta:
            out["dM"] = self.dM[:self.M.size]
            out["dD"] = self.dD[:self.ar.size]
        return out


def solve_workload(w, idx=None, tol=DEFAULT_TOL, max_iter=DEFAULT_MAX_ITER,
                   adjoint=True, threads=1, theta=False):
    """Forward (+ adjoint with the workload's g) for a packed ragged batch.

    ``idx`` restricts the work to those instances (outputs of the others stay
    zero).  Returns a dict of packed float64 outputs (a, dqfrc, daref, dJ), the
    active set (uint8, packed like aref), status and iters (int32 per
    instance).  With ``theta`` it adds dM (packed like M) and dD (packed like
    D), the remaining parameter gradients of Eq. 17.
    """
    pw = PreparedWorkload(w, tol=tol, max_iter=max_iter, adjoint=adjoint, theta=theta)
    if idx is None:
        pw.run_all(threads=threads)
    else:
        sel = [int(b) for b in np.asarray(idx).ravel()]
        if threads <= 1 or len(sel) <= 1:
            for b in sel:
                pw.run(b, b + 1)
        else:
            parts = [p for p in np.array_split(np.asarray(sel), threads) if len(p)]

            def worker(bs):
                for b in bs:
                    pw.run(int(b), int(b) + 1)

            ts = [threading.Thread(target=worker, args=(p,)) for p in parts]
            for t in ts:
                t.start()
            for t in ts:
                t.join()
    return pw.outputs()
