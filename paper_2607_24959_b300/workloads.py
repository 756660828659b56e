"""Seeded synthetic inputs for the batched contact solve.

This module only draws random problem data and packs it into the flat ragged
layout that the C ABI takes (``include/contact_solve.h``).  It holds none of the
solver's arithmetic, so both the CUDA path and the FP64 oracle can be fed from
it without sharing any method code.

Problem data per instance (Section III-A, Eqs. 1 and 5 with the pyramidal
reading of the cone term):

* ``M``    nv x nv symmetric positive definite mass matrix (row-major),
* ``J``    m x nv constraint Jacobian, m = 4 * contacts (4 pyramid rows each),
* ``qfrc`` nv smooth generalised force (tau - c in Eq. 1),
* ``aref`` m reference accelerations,
* ``D``    m positive row stiffnesses (D = R^-1 in Eq. 4),
* ``g``    nv loss cotangent dL/da (loss L = g^T a),
* ``mu``   (round-cone workloads only) m friction coefficients, one value per
           contact repeated on its three rows.

Round (elliptic) cone workloads use three rows per contact (normal, two
tangents); D holds D_N on the normal row and one tangential D_T on both
tangent rows, and mu_c ~ U(0.2, 1.2).

Distributions: J, qfrc, aref, g ~ N(0,1); D_i = 10^U(2,5).  M is either
``L L^T + 0.1 I`` with Gaussian L (the tiny workload) or ``Q diag(lambda) Q^T``
with Q Haar-orthogonal and lambda log-spaced in [1, cond] (a set condition
number).  Values are drawn in float64 and rounded once to float32; the float32
numbers are the problem (the oracle receives them widened exactly).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Mirrors ``cs_inst`` in include/contact_solve.h (40 bytes, little-endian).
INST_DTYPE = np.dtype(
    [("nv", "<i4"), ("m", "<i4"), ("off_M", "<i8"), ("off_J", "<i8"),
     ("off_v", "<i8"), ("off_r", "<i8")]
)

ROWS_PER_CONTACT = 4


def _align4(x: int) -> int:
    return (int(x) + 3) & ~3


@dataclasses.dataclass
class Workload:
    """A packed ragged batch on the host (float32 arrays + instance table)."""

    name: str
    inst: np.ndarray          # INST_DTYPE[n]
    M: np.ndarray             # float32[total_M]
    J: np.ndarray             # float32[total_J]
    qfrc: np.ndarray          # float32[total_v]
    aref: np.ndarray          # float32[total_r]
    D: np.ndarray             # float32[total_r]
    g: np.ndarray             # float32[total_v]
    params: dict
    mu: np.ndarray | None = None  # float32[total_r], round-cone workloads only

    @property
    def n(self) -> int:
        return int(self.inst.shape[0])

    @property
    def nv_max(self) -> int:
        return int(self.inst["nv"].max()) if self.n else 0

    @property
    def m_max(self) -> int:
        return int(self.inst["m"].max()) if self.n else 0

    def instance(self, b: int) -> dict:
        """Per-instance views (float32) of instance ``b``."""
        e = self.inst[b]
        nv, m = int(e["nv"]), int(e["m"])
        oM, oJ, ov, orr = (int(e["off_M"]), int(e["off_J"]), int(e["off_v"]),
                           int(e["off_r"]))
        out = dict(
            nv=nv, m=m,
            M=self.M[oM:oM + nv * nv].reshape(nv, nv),
            J=self.J[oJ:oJ + m * nv].reshape(m, nv),
            qfrc=self.qfrc[ov:ov + nv], aref=self.aref[orr:orr + m],
            D=self.D[orr:orr + m], g=self.g[ov:ov + nv],
        )
        if self.mu is not None:
            out["mu"] = self.mu[orr:orr + m]
        return out

    def subset(self, idx) -> "Workload":
        """Re-pack the instances ``idx`` (in that order) into a new workload."""
        parts = [self.instance(int(b)) for b in idx]
        return pack(parts, name=f"{self.name}[subset]", params=dict(self.params))


def layout(nvs, ms):
    """Offsets for instances with sizes (nv_b, m_b), each block 16-byte aligned.

    Returns (inst table, total_M, total_J, total_v, total_r).
    """
    nvs = np.asarray(nvs, dtype=np.int64)
    ms = np.asarray(ms, dtype=np.int64)
    n = nvs.shape[0]
    inst = np.zeros(n, dtype=INST_DTYPE)
    sM = np.array([_align4(v * v) for v in nvs], dtype=np.int64)
    sJ = np.array([_align4(mm * v) for mm, v in zip(ms, nvs)], dtype=np.int64)
    sv = np.array([_align4(v) for v in nvs], dtype=np.int64)
    sr = np.array([_align4(mm) for mm in ms], dtype=np.int64)

    def excl(s):
        o = np.zeros(n, dtype=np.int64)
        if n > 1:
            o[1:] = np.cumsum(s)[:-1]
        return o

    inst["nv"] = nvs
    inst["m"] = ms
    inst["off_M"] = excl(sM)
    inst["off_J"] = excl(sJ)
    inst["off_v"] = excl(sv)
    inst["off_r"] = excl(sr)
    return inst, int(sM.sum()), int(sJ.sum()), int(sv.sum()), int(sr.sum())


def pack(parts, name="custom", params=None) -> Workload:
    """Pack a list of per-instance dicts (M, J, qfrc, aref, D, g) into a batch."""
    nvs = [int(np.asarray(p["M"]).shape[0]) for p in parts]
    ms = [int(np.asarray(p["J"]).reshape(-1, nv).shape[0]) if nv else 0
          for p, nv in zip(parts, nvs)]
    inst, tM, tJ, tv, tr = layout(nvs, ms)
    M = np.zeros(tM, np.float32)
    J = np.zeros(tJ, np.float32)
    qfrc = np.zeros(tv, np.float32)
    g = np.zeros(tv, np.float32)
    aref = np.zeros(tr, np.float32)
    D = np.zeros(tr, np.float32)
    has_mu = bool(parts) and all("mu" in p for p in parts)
    mu = np.zeros(tr, np.float32) if has_mu else None
    for b, p in enumerate(parts):
        e = inst[b]
        nv, m = int(e["nv"]), int(e["m"])
        oM, oJ, ov, orr = (int(e["off_M"]), int(e["off_J"]), int(e["off_v"]),
                           int(e["off_r"]))
        M[oM:oM + nv * nv] = np.asarray(p["M"], np.float32).ravel()
        J[oJ:oJ + m * nv] = np.asarray(p["J"], np.float32).ravel()
        qfrc[ov:ov + nv] = np.asarray(p["qfrc"], np.float32)
        g[ov:ov + nv] = np.asarray(p.get("g", np.zeros(nv)), np.float32)
        aref[orr:orr + m] = np.asarray(p["aref"], np.float32)
        D[orr:orr + m] = np.asarray(p["D"], np.float32)
        if has_mu:
            mu[orr:orr + m] = np.asarray(p["mu"], np.float32)
    return Workload(name, inst, M, J, qfrc, aref, D, g, params or {}, mu)


def _mass_matrices(rng, n, nv, kind, cond):
    """n SPD matrices (float64), symmetrised so the float32 cast stays symmetric."""
    if kind == "wishart":
        L = rng.standard_normal((n, nv, nv))
        M = L @ np.swapaxes(L, 1, 2) + 0.1 * np.eye(nv)
    elif kind == "spectrum":
        G = rng.standard_normal((n, nv, nv))
        Q, R = np.linalg.qr(G)
        Q = Q * np.sign(np.diagonal(R, axis1=1, axis2=2))[:, None, :]
        lam = np.logspace(0.0, math.log10(cond), nv) if nv > 1 else np.ones(1)
        M = (Q * lam[None, None, :]) @ np.swapaxes(Q, 1, 2)
    else:
        raise ValueError(kind)
    return 0.5 * (M + np.swapaxes(M, 1, 2))


def generate(name, n, nv, contacts, *, seed, m_kind="spectrum", cond=1e3,
             d_lo=2.0, d_hi=5.0, cone="pyramid", mu_lo=0.2, mu_hi=1.2) -> Workload:
    """Draw ``n`` instances with fixed ``nv`` and per-instance contact counts.

    ``contacts`` is an int (every instance) or an array of length n.
    ``cone`` is "pyramid" (four rows per contact) or "elliptic" (three rows
    per contact with per-contact D_N, D_T and mu).
    """
    if cone not in ("pyramid", "elliptic"):
        raise ValueError(cone)
    rng = np.random.Generator(np.random.PCG64(seed))
    nc = np.broadcast_to(np.asarray(contacts, dtype=np.int64), (n,)).copy()
    ms = (ROWS_PER_CONTACT if cone == "pyramid" else 3) * nc
    inst, tM, tJ, tv, tr = layout(np.full(n, nv), ms)
    Ms = _mass_matrices(rng, n, nv, m_kind, cond).astype(np.float32)
    total_rows = int(ms.sum())
    Jrows = rng.standard_normal((total_rows, nv)).astype(np.float32)
    qf = rng.standard_normal((n, nv)).astype(np.float32)
    ar = rng.standard_normal(total_rows).astype(np.float32)
    Dv = (10.0 ** rng.uniform(d_lo, d_hi, total_rows)).astype(np.float32)
    gv = rng.standard_normal((n, nv)).astype(np.float32)

    M = np.zeros(tM, np.float32)
    J = np.zeros(tJ, np.float32)
    qfrc = np.zeros(tv, np.float32)
    g = np.zeros(tv, np.float32)
    aref = np.zeros(tr, np.float32)
    D = np.zeros(tr, np.float32)
    # Vectorised scatter into the aligned packed layout.
    oM = inst["off_M"][:, None] + np.arange(nv * nv)[None, :]
    M[oM.ravel()] = Ms.reshape(n, -1).ravel()
    ov = inst["off_v"][:, None] + np.arange(nv)[None, :]
    qfrc[ov.ravel()] = qf.ravel()
    g[ov.ravel()] = gv.ravel()
    row_start = np.zeros(n, np.int64)
    if n > 1:
        row_start[1:] = np.cumsum(ms)[:-1]
    inst_of_row = np.repeat(np.arange(n), ms)
    local_row = np.arange(total_rows) - row_start[inst_of_row]
    rdst = inst["off_r"][inst_of_row] + local_row
    aref[rdst] = ar
    D[rdst] = Dv
    jdst = (inst["off_J"][inst_of_row] + local_row * nv)[:, None] + np.arange(nv)[None, :]
    J[jdst.ravel()] = Jrows.ravel()
    params = dict(n=n, nv=nv, seed=seed, m_kind=m_kind, cond=cond,
                  d_range=(10 ** d_lo, 10 ** d_hi), cone=cone)
    mu = None
    if cone == "elliptic":
        # drawn after everything else, so the other arrays match the draws
        # of a pyramid workload with the same seed and row count
        ncon = total_rows // 3
        Dc = (10.0 ** rng.uniform(d_lo, d_hi, (ncon, 2))).astype(np.float32)
        muc = rng.uniform(mu_lo, mu_hi, ncon).astype(np.float32)
        Drow = np.repeat(Dc, [1, 2], axis=1).reshape(-1)       # D_N, D_T, D_T
        D[rdst] = Drow
        mu = np.zeros(tr, np.float32)
        mu[rdst] = np.repeat(muc, 3)
        params["mu_range"] = (mu_lo, mu_hi)
    return Workload(name, inst, M, J, qfrc, aref, D, g, params, mu)


# The five workloads (sizes and distributions of the paper-scale settings):
#   tiny      1024 x (nv 3,  2 contacts)       M = L L^T + 0.1 I
#   franka    8192 x (nv 9,  16 contacts)      cond(M) = 1e3
#   quadruped 512 trajectories x 64 steps = 32768 x (nv 18, U{0..32} contacts),
#             cond(M) = 1e3 (headline)
#   nv96      2048 x (nv 96, 16 contacts)      cond(M) = 1e4
#   nc256     256  x (nv 18, 256 contacts)     cond(M) = 1e3
SEEDS = dict(tiny=1001, franka=1002, quadruped=1003, nv96=1004, nc256=1004,
             serve=1005)


def tiny(n=1024, seed=SEEDS["tiny"]):
    return generate("tiny", n, 3, 2, seed=seed, m_kind="wishart")


def franka(n=8192, seed=SEEDS["franka"]):
    return generate("franka", n, 9, 16, seed=seed, cond=1e3)


def quadruped(n=32768, seed=SEEDS["quadruped"], max_contacts=32):
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    nc = rng.integers(0, max_contacts + 1, size=n)
    return generate("quadruped", n, 18, nc, seed=seed, cond=1e3)


def nv96(n=2048, seed=SEEDS["nv96"]):
    return generate("nv96", n, 96, 16, seed=seed, cond=1e4)


def nc256(n=256, seed=SEEDS["nc256"] + 1):
    return generate("nc256", n, 18, 256, seed=seed, cond=1e3)


def quadruped_elliptic(n=32768, seed=SEEDS["quadruped"], max_contacts=32):
    """The quadruped batch with MuJoCo's round cone: three rows per contact."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    nc = rng.integers(0, max_contacts + 1, size=n)
    return generate("quadruped_elliptic", n, 18, nc, seed=seed, cond=1e3, cone="elliptic")


def franka_elliptic(n=8192, seed=SEEDS["franka"]):
    return generate("franka_elliptic", n, 9, 16, seed=seed, cond=1e3, cone="elliptic")


def serve_stream(n_requests=200_000, rate=50_000.0, seed=SEEDS["serve"],
                 nv_choices=(3, 9, 18, 96), nv_probs=(0.3, 0.3, 0.3, 0.1),
                 max_contacts=64):
    """Request stream: arrival times (s), nv and contact count per request.

    Arrivals are Poisson (exponential inter-arrival at ``rate`` req/s).  The
    per-request data are drawn later by ``serve_request(i)`` from a
    per-request seed, so a request's data do not depend on the mix.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    nv = rng.choice(np.asarray(nv_choices), size=n_requests, p=np.asarray(nv_probs))
    nc = rng.integers(0, max_contacts + 1, size=n_requests)
    return t, nv.astype(np.int64), nc.astype(np.int64)


def serve_request(i, nv, nc, seed=SEEDS["serve"]):
    """Data of request ``i`` (one instance), independent of any other request."""
    cond = 1e4 if nv >= 96 else 1e3
    w = generate("serve", 1, int(nv), int(nc), seed=seed * 1_000_003 + int(i),
                 cond=cond)
    return w.instance(0)
