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
_LIB = os.path.join(_HERE, "_cs_oracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "OK", 1: "MAXITER", 2: "CHOLFAIL", 3: "NONFINITE", 4: "BADSHAPE",
          5: "NOPROGRESS"}
DEFAULT_TOL = 1e-12
DEFAULT_MAX_ITER = 100


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2, no fast-math) if it is missing or stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", _SRC,
                           "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


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


def solve_workload(w, idx=None, tol=DEFAULT_TOL, max_iter=DEFAULT_MAX_ITER,
                   adjoint=True, threads=1, theta=False):
    """Forward (+ adjoint with the workload's g) for a packed ragged batch.

    ``idx`` restricts the work to those instances (outputs of the others stay
    zero).  Returns a dict of packed float64 outputs (a, dqfrc, daref, dJ), the
    active set (uint8, packed like aref), status and iters (int32 per
    instance).  With ``theta`` it adds dM (packed like M) and dD (packed like
    D), the remaining parameter gradients of Eq. 17.
    """
    lib = _load()
    inst = w.inst
    n = inst.shape[0]
    nv = np.ascontiguousarray(inst["nv"], np.int32)
    m = np.ascontiguousarray(inst["m"], np.int32)
    offs = [np.ascontiguousarray(inst[k], np.int64)
            for k in ("off_M", "off_J", "off_v", "off_r")]
    M, J, q, ar, D, g = (np.ascontiguousarray(x, np.float64)
                         for x in (w.M, w.J, w.qfrc, w.aref, w.D, w.g))
    a = np.zeros(max(q.size, 1))
    dq = np.zeros(max(q.size, 1))
    dr = np.zeros(max(ar.size, 1))
    dJ = np.zeros(max(J.size, 1))
    act = np.zeros(max(ar.size, 1), np.uint8)
    dM = np.zeros(max(M.size, 1)) if theta else None
    dD = np.zeros(max(ar.size, 1)) if theta else None
    status = np.full(n, -1, np.int32)
    iters = np.zeros(n, np.int32)
    P = ctypes.POINTER
    cd = lambda x: x.ctypes.data_as(P(ctypes.c_double))
    ci32 = lambda x: x.ctypes.data_as(P(ctypes.c_int32))
    ci64 = lambda x: x.ctypes.data_as(P(ctypes.c_int64))

    def run(lo, hi):
        lib.oracle_batch(lo, hi, ci32(nv), ci32(m), *[ci64(o) for o in offs],
                         cd(M), cd(J), cd(q), cd(ar), cd(D),
                         cd(g) if adjoint else None, tol, max_iter, cd(a),
                         act.ctypes.data_as(P(ctypes.c_uint8)), ci32(status),
                         ci32(iters), cd(dq), cd(dr), cd(dJ),
                         cd(dM) if theta else None, cd(dD) if theta else None)

    if idx is None:
        ranges = []
        chunk = max(1, (n + threads - 1) // max(threads, 1))
        for lo in range(0, n, chunk):
            ranges.append((lo, min(n, lo + chunk)))
    else:
        ranges = [(int(b), int(b) + 1) for b in np.asarray(idx).ravel()]
    if threads <= 1 or len(ranges) <= 1:
        for lo, hi in ranges:
            run(lo, hi)
    else:
        # ctypes releases the GIL during the C call, so plain threads give
        # real parallelism over disjoint instance ranges.
        if idx is not None:
            parts = np.array_split(np.arange(len(ranges)), threads)
            work = [[ranges[i] for i in p] for p in parts if len(p)]
        else:
            work = [[r] for r in ranges]

        def worker(rs):
            for lo, hi in rs:
                run(lo, hi)

        ts = [threading.Thread(target=worker, args=(rs,)) for rs in work]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
    out = dict(a=a[:q.size], dqfrc=dq[:q.size], daref=dr[:ar.size],
               dJ=dJ[:J.size], act=act[:ar.size], status=status, iters=iters)
    if theta:
        out["dM"] = dM[:M.size]
        out["dD"] = dD[:ar.size]
    return out
