"""Writes tiny_exact.json: exact solutions of small seeded contact problems.

For each case the minimiser of the regularised contact objective (Eq. 5,
pyramidal rows) is found by enumerating every active set S, solving the
stationarity condition with S fixed (Eq. 7 with the Newton matrix of Eq. 9),
(M + J_S^T D_S J_S) a = qfrc + J_S^T D_S aref_S, and keeping the unique S whose
signs of jar = J a - aref agree with it (strict convexity makes it unique).
The IFT adjoint of L = g^T a (Eq. 17) follows: w = H_S^-1 g, dL/dqfrc = w,
dL/daref = D_S (J w), dL/dJ = -(f w^T + (D_S J w) a^T) with
f = D min(jar, 0).  Everything is exact rational arithmetic on the float32
inputs (exact binary fractions); the stored floats are the correctly rounded
float64 values of the exact results.  Inputs come from the seeded generators
of paper_2607_24959_b300.workloads; no solver code (neither the oracle nor the
CUDA path) is used.

Run from the repository root:  python tests/golden/make_golden.py
"""
import itertools
import json
import os
import sys
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from paper_2607_24959_b300 import workloads as W  # noqa: E402


def _solve(A, b):
    """Gauss-Jordan elimination in exact arithmetic (A nonsingular)."""
    n = len(b)
    A = [row[:] + [b[i]] for i, row in enumerate(A)]
    for c in range(n):
        piv = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        for r in range(n):
            if r != c and A[r][c] != 0:
                fct = A[r][c] / A[c][c]
                A[r] = [x - fct * y for x, y in zip(A[r], A[c])]
    return [A[i][n] / A[i][i] for i in range(n)]


def exact_case(M, J, q, ar, D, g):
    F = lambda x: Fraction(float(x))  # noqa: E731
    nv, m = len(M), len(J)
    Mx = [[F(x) for x in row] for row in M]
    Jx = [[F(x) for x in row] for row in J]
    qx, arx, Dx, gx = ([F(x) for x in v] for v in (q, ar, D, g))
    found = []
    for S in itertools.product([0, 1], repeat=m):
        H = [[Mx[j][k] + sum(Dx[i] * Jx[i][j] * Jx[i][k] for i in range(m) if S[i])
              for k in range(nv)] for j in range(nv)]
        rhs = [qx[j] + sum(Jx[i][j] * Dx[i] * arx[i] for i in range(m) if S[i])
               for j in range(nv)]
        a = _solve(H, rhs)
        jar = [sum(Jx[i][k] * a[k] for k in range(nv)) - arx[i] for i in range(m)]
        if all((jar[i] < 0) == bool(S[i]) for i in range(m)):
            found.append((S, H, a, jar))
    assert len(found) == 1, f"{len(found)} consistent active sets"
    S, H, a, jar = found[0]
    w = _solve(H, gx)
    jw = [sum(Jx[i][k] * w[k] for k in range(nv)) for i in range(m)]
    daref = [Dx[i] * jw[i] if S[i] else Fraction(0) for i in range(m)]
    f = [Dx[i] * jar[i] if jar[i] < 0 else Fraction(0) for i in range(m)]
    dJ = [[-(f[i] * w[k] + daref[i] * a[k]) for k in range(nv)] for i in range(m)]
    # distance of the nearest row from its boundary, relative to its scale
    scale = [sum(abs(Jx[i][k] * a[k]) for k in range(nv)) + abs(arx[i]) for i in range(m)]
    margin = min((abs(jar[i]) / scale[i] for i in range(m)), default=Fraction(1))
    fl = lambda v: [float(x) for x in v]  # noqa: E731
    return dict(active=[int(s) for s in S], a=fl(a), dqfrc=fl(w), daref=fl(daref),
                dJ=[fl(r) for r in dJ], margin=float(margin))


def case_from(p, name):
    M, J = np.asarray(p["M"]), np.asarray(p["J"])
    ins = dict(M=M.tolist(), J=J.tolist(), qfrc=np.asarray(p["qfrc"]).tolist(),
               aref=np.asarray(p["aref"]).tolist(), D=np.asarray(p["D"]).tolist(),
               g=np.asarray(p["g"]).tolist())
    out = exact_case(ins["M"], ins["J"], ins["qfrc"], ins["aref"], ins["D"], ins["g"])
    return dict(name=name, nv=int(M.shape[0]), m=int(J.shape[0]), **ins, **out)


def build_document():
    cases = []
    # hand-worked two-DoF case: a = (-5/11, 12/11), w = (4/11, -3/11),
    # daref = 3/11, dJ = (63/121, -72/121)
    hand = dict(M=np.diag([2.0, 1.0]), J=np.array([[1.0, 1.0]]), qfrc=[-2.0, 0.0],
                aref=[1.0], D=[3.0], g=[1.0, 0.0])
    cases.append(case_from(hand, "two-dof"))
    sets = [("tiny", W.tiny(n=10, seed=4242)),
            ("nv5", W.generate("nv5", 4, 5, 2, seed=4243, cond=1e2)),
            ("nv2-one-contact", W.generate("nv2", 4, 2, 1, seed=4244, cond=1e1)),
            ("no-contact", W.generate("nc0", 2, 4, 0, seed=4245, cond=1e2))]
    # contacts present but every row inactive (aref far below J a0)
    p = W.tiny(n=1, seed=4246).instance(0)
    p = dict(p, aref=np.asarray(p["aref"], np.float32) - np.float32(1000.0))
    cases.append(case_from(p, "all-rows-inactive"))
    for label, w in sets:
        for b in range(w.n):
            c = case_from(w.instance(b), f"{label}-{b}")
            if c["margin"] >= 1e-4:  # keep instances with no row near its boundary
                cases.append(c)
    return {
        "what": "exact minimisers of Eq. 5 (pyramidal rows) and their Eq. 17 adjoints "
                "for L = g^T a, by exact-rational enumeration of active sets",
        "written_by": "tests/golden/make_golden.py (no solver code used)",
        "citation": "Eq. 5 (objective), Eq. 7 (stationarity), Eq. 9 (Newton matrix), "
                    "Eq. 17 (IFT adjoint)",
        "cases": cases,
    }


def main():
    doc = build_document()
    cases = doc["cases"]
    out = os.path.join(HERE, "tiny_exact.json")
    with open(out, "w") as fh:
        json.dump(doc, fh, indent=0)
    print(f"wrote {len(cases)} cases to {out}")


if __name__ == "__main__":
    main()
