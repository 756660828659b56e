"""Pins of the FP64 oracle against things other than itself.

Each test fixes part of the oracle with a result the paper and the mathematics
determine independently of its code:

* closed forms: nc = 0 (Eq. 1: a = M^-1 qfrc, w = M^-1 g) and a single row
  (Sherman-Morrison on Eq. 9), plus a hand-worked two-DoF example;
* brute force: every active set of an m <= 8 problem, solved in exact rational
  arithmetic and in float64, keeping the unique set consistent with the signs
  of jar (strict convexity of Eq. 5 makes it unique);
* the line search against a dense evaluation of phi (Eqs. 5, 10);
* central finite differences of L = g^T a* with an epsilon sweep and the
  active set held fixed (the paper's validation method, Section III-E), for
  every parameter (qfrc, aref, J, and M, D through the full Eq. 17);
* an independently written unrolled Newton solve differentiated by torch
  autograd, which must equal the IFT adjoint once the active set has settled
  (Eqs. 13-14) and differ from it when truncated early;
* invariants: r(a*) = 0 (Eq. 7), positive homogeneity, start-point
  independence (Eq. 14), row-permutation equivariance, the K cap, error codes.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from paper_2607_24959_b300 import workloads as W


def _f64(p):
    return {k: (np.asarray(v, np.float64) if not isinstance(v, int) else v)
            for k, v in p.items()}


def _solve(p, **kw):
    return oracle.solve_one(p["M"], p["J"], p["qfrc"], p["aref"], p["D"], **kw)


def _adj(p, a):
    return oracle.adjoint_one(p["M"], p["J"], p["qfrc"], p["aref"], p["D"], a,
                              p["g"])


def _rel(x, y):
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    if x.size == 0:
        return 0.0
    return float(np.max(np.abs(x - y)) / max(np.max(np.abs(y)), 1e-300))


# ---------------------------------------------------------------- closed forms

def test_no_contacts_closed_form():
    """nc = 0: a* = M^-1 qfrc (Eq. 1), adjoint w = M^-1 g (Eq. 17 with H = M)."""
    w = W.generate("nc0", 20, 9, 0, seed=11, cond=1e3)
    for b in range(w.n):
        p = _f64(w.instance(b))
        a, act, st, it = _solve(p)
        assert st == 0 and it == 0 and act.size == 0
        assert _rel(a, np.linalg.solve(p["M"], p["qfrc"])) < 1e-12
        dq, dr, dJ, _, st2 = _adj(p, a)
        assert st2 == 0 and dr.size == 0 and dJ.size == 0
        assert _rel(dq, np.linalg.solve(p["M"], p["g"])) < 1e-12


def _one_row_closed_form(M, j, aref, D, qfrc, g):
    """Sherman-Morrison solution of the one-row problem (Eqs. 5, 9, 17)."""
    Minv_j = np.linalg.solve(M, j)
    a0 = np.linalg.solve(M, qfrc)
    c = j @ Minv_j
    jar0 = j @ a0 - aref
    Minv_g = np.linalg.solve(M, g)
    if jar0 >= 0:
        return a0, False, Minv_g, 0.0, np.zeros_like(j)
    jar = jar0 / (1.0 + D * c)
    a = a0 - D * jar * Minv_j
    f = D * jar
    w = Minv_g - (D * (j @ Minv_g) / (1.0 + D * c)) * Minv_j
    daref = D * (j @ w)
    dJ = -(f * w + daref * a)
    return a, True, w, daref, dJ


def test_single_row_closed_form():
    rng = np.random.default_rng(5)
    n_active = 0
    for trial in range(200):
        nv = int(rng.integers(1, 8))
        G = rng.standard_normal((nv, nv))
        M = G @ G.T + 0.5 * np.eye(nv)
        j = rng.standard_normal(nv)
        aref = float(rng.standard_normal())
        D = float(10 ** rng.uniform(2, 5))
        qfrc = rng.standard_normal(nv)
        g = rng.standard_normal(nv)
        a_cf, act_cf, w_cf, dr_cf, dJ_cf = _one_row_closed_form(M, j, aref, D,
                                                                qfrc, g)
        a, act, st, _ = oracle.solve_one(M, j[None, :], qfrc, [aref], [D])
        assert st == 0
        assert bool(act[0]) == act_cf
        n_active += act_cf
        assert _rel(a, a_cf) < 1e-10
        dq, dr, dJ, _, _ = oracle.adjoint_one(M, j[None, :], qfrc, [aref], [D],
                                              a, g)
        assert _rel(dq, w_cf) < 1e-9
        assert abs(dr[0] - dr_cf) <= 1e-8 * max(1.0, abs(dr_cf))
        assert _rel(dJ[0], dJ_cf) < 1e-8 or np.max(np.abs(dJ_cf)) == 0
    assert 40 < n_active < 160


def test_single_row_theta_closed_form():
    """dL/dD and dL/dM of the one-row problem from the closed-form solution.

    With c = j^T M^-1 j and jar0 = j^T a0 - aref < 0, the solution is
    a*(D) = a0 - (D jar0 / (1 + D c)) M^-1 j, so dL/dD = g^T da*/dD =
    -(g^T M^-1 j) jar0 / (1 + D c)^2.  For M, a*(M) is differentiated along a
    symmetric direction E by the product rule on that same expression
    (d M^-1 = -M^-1 E M^-1), giving a value to compare with <dM, E>."""
    rng = np.random.default_rng(15)
    n_active = 0
    for trial in range(200):
        nv = int(rng.integers(1, 8))
        G = rng.standard_normal((nv, nv))
        M = G @ G.T + 0.5 * np.eye(nv)
        j = rng.standard_normal(nv)
        aref = float(rng.standard_normal())
        D = float(10 ** rng.uniform(2, 5))
        qfrc = rng.standard_normal(nv)
        g = rng.standard_normal(nv)
        a, act, st, _ = oracle.solve_one(M, j[None, :], qfrc, [aref], [D])
        assert st == 0
        _, _, _, dM, dD, _, st2 = oracle.adjoint_theta_one(
            M, j[None, :], qfrc, [aref], [D], a, g)
        assert st2 == 0
        Mi = np.linalg.inv(M)
        a0 = Mi @ qfrc
        mj = Mi @ j
        c = j @ mj
        jar0 = j @ a0 - aref
        E = rng.standard_normal((nv, nv))
        E = E + E.T
        dMi = -Mi @ E @ Mi            # derivative of M^-1 along E
        da0 = dMi @ qfrc
        if jar0 < 0:
            n_active += 1
            dD_cf = -(g @ mj) * jar0 / (1.0 + D * c) ** 2
            dmj = dMi @ j
            dc = j @ dmj
            djar0 = j @ da0
            coef = D * jar0 / (1.0 + D * c)
            dcoef = D * djar0 / (1.0 + D * c) - D * jar0 * D * dc / (1.0 + D * c) ** 2
            da = da0 - dcoef * mj - coef * dmj
        else:
            dD_cf = 0.0
            da = da0
        assert abs(dD[0] - dD_cf) <= 1e-9 * max(abs(dD_cf), 1e-12) + 1e-15
        dirn = g @ da
        assert abs(np.sum(dM * E) - dirn) <= 1e-9 * max(1.0, abs(dirn))
        assert np.allclose(dM, dM.T, rtol=0, atol=0)
    assert 40 < n_active < 160


def test_hand_worked_two_dof():
    """M = diag(2,1), J = [1 1], aref = 1, D = 3, qfrc = (-2,0), g = (1,0).

    a0 = (-1, 0) gives jar = -2 < 0, so the row is active; then
    H = [[5,3],[3,4]], a = H^-1 (qfrc + J^T D aref) = (-5/11, 12/11) with
    jar = -4/11 < 0 (consistent).  w = H^-1 g = (4/11, -3/11), daref = D J w =
    3/11, f = D jar = -12/11, dJ = -(f w^T + daref a^T) = (63/121, -72/121).
    """
    M = np.diag([2.0, 1.0])
    J = np.array([[1.0, 1.0]])
    a, act, st, _ = oracle.solve_one(M, J, [-2.0, 0.0], [1.0], [3.0])
    assert st == 0 and act.tolist() == [True]
    assert np.allclose(a, [-5 / 11, 12 / 11], rtol=0, atol=1e-15)
    dq, dr, dJ, _, _ = oracle.adjoint_one(M, J, [-2.0, 0.0], [1.0], [3.0], a,
                                          [1.0, 0.0])
    assert np.allclose(dq, [4 / 11, -3 / 11], rtol=0, atol=1e-15)
    assert np.allclose(dr, [3 / 11], rtol=0, atol=1e-15)
    assert np.allclose(dJ, [[63 / 121, -72 / 121]], rtol=0, atol=1e-15)


# ----------------------------------------------------------------- brute force

def _brute_force_f64(p):
    """All 2^m active sets; keep the one consistent with sign(jar)."""
    M, J, q, ar, D = p["M"], p["J"], p["qfrc"], p["aref"], p["D"]
    m, nv = J.shape
    found = []
    for bits in range(1 << m):
        S = np.array([(bits >> i) & 1 for i in range(m)], bool)
        H = M + (J[S].T * D[S]) @ J[S]
        a = np.linalg.solve(H, q + J[S].T @ (D[S] * ar[S]))
        jar = J @ a - ar
        if np.all(jar[S] < 0) and np.all(jar[~S] >= 0):
            found.append((a, S, jar))
    return found


def _solve_exact(A, b):
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


def _brute_force_exact(p):
    """Same enumeration in exact rational arithmetic (inputs are float32,
    hence exact binary fractions)."""
    F = lambda x: Fraction(float(x))
    M = [[F(x) for x in row] for row in p["M"]]
    J = [[F(x) for x in row] for row in p["J"]]
    q = [F(x) for x in p["qfrc"]]
    ar = [F(x) for x in p["aref"]]
    D = [F(x) for x in p["D"]]
    m, nv = len(J), len(M)
    sols = []
    for S in itertools.product([0, 1], repeat=m):
        H = [[M[j][k] + sum(D[i] * J[i][j] * J[i][k] for i in range(m) if S[i])
              for k in range(nv)] for j in range(nv)]
        rhs = [q[j] + sum(J[i][j] * D[i] * ar[i] for i in range(m) if S[i])
               for j in range(nv)]
        a = _solve_exact(H, rhs)
        jar = [sum(J[i][k] * a[k] for k in range(nv)) - ar[i] for i in range(m)]
        if all((jar[i] < 0) == bool(S[i]) for i in range(m)):
            sols.append((a, S))
    return sols


def test_brute_force_exact_rational():
    w = W.tiny(6)
    for b in range(w.n):
        p = _f64(w.instance(b))
        sols = _brute_force_exact(p)
        assert len(sols) == 1, "strict convexity gives a unique consistent set"
        a_ex, S = sols[0]
        a, act, st, _ = _solve(p)
        assert st == 0
        assert act.tolist() == [bool(s) for s in S]
        assert _rel(a, [float(x) for x in a_ex]) < 1e-12


def test_brute_force_whole_tiny_workload():
    """The whole tiny workload (1024 x nv 3, m 8): unique consistent set,
    matched by the oracle's active set and acceleration."""
    w = W.tiny()
    out = oracle.solve_workload(w, adjoint=False)
    assert np.all(out["status"] == 0)
    for b in range(w.n):
        p = _f64(w.instance(b))
        found = _brute_force_f64(p)
        assert len(found) == 1
        a_bf, S, _ = found[0]
        e = w.inst[b]
        a = out["a"][e["off_v"]:e["off_v"] + 3]
        act = out["act"][e["off_r"]:e["off_r"] + 8].astype(bool)
        assert np.array_equal(act, S)
        assert _rel(a, a_bf) < 1e-10


# ---------------------------------------------------------------- line search

def test_line_search_is_exact_minimiser():
    w = W.franka(64)
    rng = np.random.default_rng(3)
    for b in range(w.n):
        p = _f64(w.instance(b))
        a = np.linalg.solve(p["M"], p["qfrc"]) + 0.3 * rng.standard_normal(9)
        r, f, act, _ = oracle.residual_one(p["M"], p["J"], p["qfrc"], p["aref"],
                                           p["D"], a)
        H = p["M"] + (p["J"][act].T * p["D"][act]) @ p["J"][act]
        d = -np.linalg.solve(H, r)
        alpha = oracle.line_search_one(p["M"], p["J"], p["qfrc"], p["aref"],
                                       p["D"], a, d)
        assert alpha > 0
        phi = lambda t: oracle.objective_one(p["M"], p["J"], p["qfrc"],
                                             p["aref"], p["D"], a + t * d)
        # phi'(alpha) = d^T r(a + alpha d) must vanish at the exact minimiser.
        r2, _, _, sc = oracle.residual_one(p["M"], p["J"], p["qfrc"], p["aref"],
                                           p["D"], a + alpha * d)
        assert abs(d @ r2) <= 1e-9 * sc * np.abs(d).sum()
        grid = alpha * np.linspace(0.0, 3.0, 61)
        vals = np.array([phi(t) for t in grid])
        assert phi(alpha) <= vals.min() + 1e-9 * max(1.0, abs(vals.min()))


# ------------------------------------------------------- finite differences

def _loss(p, key, idx, delta):
    q = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in p.items()}
    q[key].reshape(-1)[idx] += delta
    a, act, st, _ = _solve(q)
    assert st == 0
    return float(q["g"] @ a), act


def test_central_differences_with_epsilon_sweep():
    """dL/dqfrc, dL/daref, dL/dJ of Eq. 17 against central FD of the oracle's
    own forward solve, the active set held fixed under every perturbation."""
    w = W.tiny(12)
    skipped = checked = 0
    for b in range(w.n):
        p = _f64(w.instance(b))
        a, act, st, _ = _solve(p)
        dq, dr, dJ, _, _ = _adj(p, a)
        for key, grad in (("qfrc", dq), ("aref", dr), ("J", dJ)):
            g = grad.reshape(-1)
            for idx in range(g.size):
                ests = {}
                for h in (1e-4, 1e-5, 1e-6, 1e-7):
                    lp, actp = _loss(p, key, idx, +h)
                    lm, actm = _loss(p, key, idx, -h)
                    if not (np.array_equal(actp, act) and np.array_equal(actm, act)):
                        ests = None
                        break
                    ests[h] = (lp - lm) / (2 * h)
                if ests is None:
                    skipped += 1
                    continue
                checked += 1
                scale = max(1.0, abs(g[idx]))
                # a stable FD reference across the sweep ...
                assert abs(ests[1e-5] - ests[1e-6]) <= 1e-6 * scale
                # ... that matches the implicit derivative
                assert abs(ests[1e-6] - g[idx]) <= 2e-7 * scale, (key, idx)
    assert checked > 20 * skipped


def test_theta_central_differences():
    """dL/dM (symmetric perturbations M + h (E_jk + E_kj)) and dL/dD
    (relative perturbations D_i e^{+-h}) against central FD of the forward
    solve, the active set held fixed."""
    skipped = checked = 0
    for w in (W.tiny(8), W.franka(3)):
        for b in range(w.n):
            p = _f64(w.instance(b))
            a, act, st, _ = _solve(p)
            _, _, _, dM, dD, _, st2 = oracle.adjoint_theta_one(
                p["M"], p["J"], p["qfrc"], p["aref"], p["D"], a, p["g"])
            assert st2 == 0
            nv = p["M"].shape[0]
            cases = []
            for j in range(nv):
                for k in range(j + 1):
                    E = np.zeros((nv, nv))
                    E[j, k] += 1.0
                    if j != k:
                        E[k, j] += 1.0
                    cases.append(("M", E, float(np.sum(dM * E))))
            for i in range(p["D"].size):
                cases.append(("D", i, float(p["D"][i] * dD[i])))
            for key, dirn, expect in cases:
                ests = {}
                for h in (1e-4, 1e-5, 1e-6):
                    vals = []
                    for sgn in (1.0, -1.0):
                        q = {k2: (v.copy() if isinstance(v, np.ndarray) else v)
                             for k2, v in p.items()}
                        if key == "M":
                            q["M"] = q["M"] + sgn * h * dirn
                        else:
                            q["D"][dirn] *= np.exp(sgn * h)
                        aa, aact, sst, _ = _solve(q)
                        assert sst == 0
                        if not np.array_equal(aact, act):
                            vals = None
                            break
                        vals.append(float(q["g"] @ aa))
                    if vals is None:
                        ests = None
                        break
                    ests[h] = (vals[0] - vals[1]) / (2 * h)
                if ests is None:
                    skipped += 1
                    continue
                checked += 1
                # h = 1e-4 balances truncation (h^2) against the solver's
                # stopping tolerance divided by h
                # (values are O(1e-5 .. 1); the absolute part covers the
                # solver's stopping noise on the smallest of them)
                assert abs(ests[1e-4] - ests[1e-5]) <= 1e-5 * abs(expect) + 1e-7
                assert abs(ests[1e-4] - expect) <= 1e-6 * abs(expect) + 1e-8, (key, dirn)
    assert checked > 20 * max(skipped, 1)


# --------------------------------------------- unrolled Newton (torch autograd)

def _unrolled_newton(M, J, q, ar, D, K):
    """Newton with exact line search, written independently of the oracle in
    torch float64 so that autograd differentiates the executed trace (the
    'unrolled AD' derivative the paper compares against)."""
    a = torch.linalg.solve(M, q)
    for _ in range(K):
        jar = J @ a - ar
        act = (jar < 0).detach()
        f = D * torch.clamp(jar, max=0.0)
        r = M @ a - q + J.T @ f
        with torch.no_grad():
            scale = max(1.0, float(q.abs().max()), float((M @ a).abs().max()),
                        float((J.T @ f).abs().max()))
            rn = float(r.abs().max())
        if rn <= 1e-13 * scale:
            break
        Dact = D * act
        H = M + J.T @ (Dact[:, None] * J)
        d = -torch.linalg.solve(H, r)
        jn = (J @ (a + d) - ar).detach()
        if torch.equal(jn < 0, act):
            a = a + d        # full step, active set unchanged: exact
            break
        s = J @ d
        # locate the segment of phi' holding its root with detached values,
        # then take alpha = -c0/c1 on that segment (differentiable).
        sd, jd, Dd = s.detach(), jar.detach(), D.detach()
        c0 = float(d.detach() @ (M @ a - q).detach()) + float((Dact * s * jar).detach().sum())
        c1 = float(d.detach() @ (M @ d).detach()) + float((Dact * s * s).detach().sum())
        seg = act.clone()
        bp = torch.where(sd != 0, -jd / sd, torch.full_like(sd, -1.0))
        order = torch.argsort(bp)
        for i in order.tolist():
            if bp[i] <= 0:
                continue
            if -c0 / c1 <= float(bp[i]):
                break
            sgn = -1.0 if bool(seg[i]) else 1.0
            seg[i] = not bool(seg[i])
            c0 += sgn * float(Dd[i] * sd[i] * jd[i])
            c1 += sgn * float(Dd[i] * sd[i] * sd[i])
        Ds = D * seg
        c0t = d @ (M @ a - q) + (Ds * s * jar).sum()
        c1t = d @ (M @ d) + (Ds * s * s).sum()
        a = a - (c0t / c1t) * d
    return a


def test_unrolled_newton_derivative_matches_ift():
    w = W.franka(16)
    n_diff_k1 = 0
    for b in range(w.n):
        p = _f64(w.instance(b))
        a, act, st, it = _solve(p)
        dq, dr, dJ, dM, dD, _, _ = oracle.adjoint_theta_one(
            p["M"], p["J"], p["qfrc"], p["aref"], p["D"], a, p["g"])
        for K, expect_equal in ((50, True), (1, False)):
            T = {k: torch.tensor(p[k], dtype=torch.float64, requires_grad=True)
                 for k in ("qfrc", "aref", "J", "M", "D")}
            gt = torch.tensor(p["g"])
            aK = _unrolled_newton(T["M"], T["J"], T["qfrc"], T["aref"], T["D"], K)
            (gt @ aK).backward()
            # autograd sees M's nv^2 entries as independent; the gradient with
            # respect to a symmetric M is the symmetric part of that one
            gM = T["M"].grad.numpy()
            errs = [_rel(T["qfrc"].grad.numpy(), dq), _rel(T["aref"].grad.numpy(), dr),
                    _rel(T["J"].grad.numpy(), dJ), _rel(0.5 * (gM + gM.T), dM),
                    _rel(T["D"].grad.numpy(), dD)]
            if expect_equal:
                assert _rel(aK.detach().numpy(), a) < 1e-11
                assert max(errs) < 1e-8, errs
            elif it > 1 and max(errs) > 1e-3:
                n_diff_k1 += 1
    # truncated unrolls (K = 1) carry a different derivative (Section III-E)
    assert n_diff_k1 >= 8


def test_unrolled_oracle_matches_autograd_of_the_trace():
    """The oracle's hand-written reverse sweep through K Newton steps equals
    torch autograd applied to the independently written unrolled solver, for
    every parameter, truncated (K = 1, 2, 3) and run to convergence."""
    for w in (W.franka(10), W.tiny(10), W.quadruped(10)):
        for b in range(w.n):
            p = _f64(w.instance(b))
            for K in (1, 2, 3, 50):
                res = oracle.unrolled_one(p["M"], p["J"], p["qfrc"], p["aref"], p["D"],
                                          p["g"], K, tol=1e-13)
                T = {k: torch.tensor(p[k], dtype=torch.float64, requires_grad=True)
                     for k in ("qfrc", "aref", "J", "M", "D")}
                aK = _unrolled_newton(T["M"], T["J"], T["qfrc"], T["aref"], T["D"], K)
                (torch.tensor(p["g"]) @ aK).backward()
                gM = T["M"].grad.numpy()
                assert _rel(res["a"], aK.detach().numpy()) < 1e-10
                for key, ref in (("dqfrc", T["qfrc"].grad), ("daref", T["aref"].grad),
                                 ("dJ", T["J"].grad), ("dD", T["D"].grad)):
                    assert _rel(res[key].reshape(-1), ref.numpy().reshape(-1)) < 1e-9, (b, K, key)
                assert _rel(res["dM"], 0.5 * (gM + gM.T)) < 1e-9, (b, K)


def test_unrolled_oracle_central_differences():
    """Central FD of a -> g^T a_K(theta) for the K-step map itself (K = 2),
    where the sweep is stable (no mask of the trace changes within +-h)."""
    w = W.tiny(12)
    checked = 0
    for b in range(w.n):
        p = _f64(w.instance(b))
        res = oracle.unrolled_one(p["M"], p["J"], p["qfrc"], p["aref"], p["D"], p["g"], 2)
        for key in ("qfrc", "aref", "J", "D"):
            grad = res["d" + key]
            flat = grad.reshape(-1)
            for idx in range(flat.size):
                est = {}
                for h in (1e-5, 1e-6):
                    vals = []
                    for sgn in (1.0, -1.0):
                        q = {k2: (v.copy() if isinstance(v, np.ndarray) else v)
                             for k2, v in p.items()}
                        q[key].reshape(-1)[idx] += sgn * h
                        r2 = oracle.unrolled_one(q["M"], q["J"], q["qfrc"], q["aref"],
                                                 q["D"], q["g"], 2)
                        vals.append(float(q["g"] @ r2["a"]))
                    est[h] = (vals[0] - vals[1]) / (2 * h)
                scale = max(1.0, abs(flat[idx]))
                if abs(est[1e-5] - est[1e-6]) > 1e-6 * scale:
                    continue              # a mask of the trace flips within h
                checked += 1
                assert abs(est[1e-6] - flat[idx]) <= 1e-6 * scale, (b, key, idx)
    assert checked > 200


def test_unrolled_derivative_approaches_ift():
    """Run to convergence, the trace derivative equals the IFT adjoint
    (Eq. 17) at the returned point; truncated at K = 1 it generally does not."""
    w = W.franka(16)
    differ = 0
    for b in range(w.n):
        p = _f64(w.instance(b))
        a, act, st, it = _solve(p)
        dq, dr, dJ, dM, dD, _, _ = oracle.adjoint_theta_one(
            p["M"], p["J"], p["qfrc"], p["aref"], p["D"], a, p["g"])
        res = oracle.unrolled_one(p["M"], p["J"], p["qfrc"], p["aref"], p["D"], p["g"], 100)
        assert res["status"] == 0 and res["steps"] == it
        assert _rel(res["a"], a) < 1e-12
        for key, ref in (("dqfrc", dq), ("daref", dr), ("dJ", dJ), ("dM", dM), ("dD", dD)):
            assert _rel(res[key], ref) < 1e-8, (b, key)
        r1 = oracle.unrolled_one(p["M"], p["J"], p["qfrc"], p["aref"], p["D"], p["g"], 1)
        differ += it > 1 and _rel(r1["dqfrc"], dq) > 1e-3
    assert differ >= 8


# ------------------------------------------------------------------ invariants

def test_residual_vanishes_and_invariants():
    w = W.quadruped(48)
    rng = np.random.default_rng(9)
    for b in range(w.n):
        p = _f64(w.instance(b))
        a, act, st, it = _solve(p)
        assert st == 0
        r, f, act2, scale = oracle.residual_one(p["M"], p["J"], p["qfrc"],
                                                p["aref"], p["D"], a)
        assert np.max(np.abs(r)) <= 1e-11 * scale          # Eq. 7
        assert np.array_equal(act2, act)
        # positive homogeneity: (c qfrc, c aref) -> c a*
        c = 3.5
        a_c, act_c, _, _ = oracle.solve_one(p["M"], p["J"], c * p["qfrc"],
                                            c * p["aref"], p["D"])
        assert _rel(a_c, c * a) < 1e-10 and np.array_equal(act_c, act)
        # start-point independence (Eq. 14): same root from a random start
        a_w, act_w, st_w, _ = _solve(p, a_init=a + rng.standard_normal(18))
        assert st_w == 0 and _rel(a_w, a) < 1e-10 and np.array_equal(act_w, act)
        # row-permutation equivariance
        if p["J"].shape[0]:
            perm = rng.permutation(p["J"].shape[0])
            a_p, act_p, _, _ = oracle.solve_one(p["M"], p["J"][perm], p["qfrc"],
                                                p["aref"][perm], p["D"][perm])
            assert _rel(a_p, a) < 1e-10 and np.array_equal(act_p, act[perm])
            dq, dr, dJ, _, _ = _adj(p, a)
            dq_p, dr_p, dJ_p, _, _ = oracle.adjoint_one(
                p["M"], p["J"][perm], p["qfrc"], p["aref"][perm], p["D"][perm],
                a_p, p["g"])
            assert _rel(dr_p, dr[perm]) < 1e-8 and _rel(dJ_p, dJ[perm]) < 1e-8


def test_iteration_cap_and_error_codes():
    w = W.quadruped(64)
    p = None
    for b in range(w.n):
        q = _f64(w.instance(b))
        _, _, _, it = _solve(q)
        if it >= 4:
            p = q
            break
    assert p is not None
    a, act, st, it = _solve(p, max_iter=1)
    assert st == 1 and it == 1                 # MAXITER, not an error
    a, act, st, it = oracle.solve_one(np.eye(2), np.zeros((0, 2)), [np.nan, 0.0],
                                      [], [])
    assert st == 3                             # NONFINITE
    a, act, st, it = oracle.solve_one(-np.eye(2), np.zeros((0, 2)), [1.0, 0.0],
                                      [], [])
    assert st == 2                             # CHOLFAIL
