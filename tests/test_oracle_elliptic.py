"""Pins of the FP64 oracle's round (elliptic) Coulomb cone, each against
something other than its own formulas:

* the per-contact cost s(u) = min over z in K* of 1/2 |u - z|^2_{R^-1}
  (Eqs. 3-5) against a general constrained minimiser (scipy SLSQP on the
  three-dimensional projection), and its gradient and Hessian against
  central differences of s and of the gradient;
* friction mu = 0 reduces the cone to the normal rows alone: the solve and
  the adjoint equal the (separately pinned) pyramidal oracle run on the
  normal rows;
* stationarity and minimality of the returned point (Eqs. 6-7): central
  differences of the objective vanish there, and random perturbations do not
  lower it;
* the line search against a dense evaluation of phi(alpha) = L(a + alpha p);
* the IFT adjoint (Eq. 17) against central differences of L = g^T a* for
  qfrc, aref, J, M (symmetric directions), D_N, D_T and mu, with every
  contact's zone held fixed.
"""
import numpy as np
import pytest
from scipy.optimize import minimize

import oracle
from paper_2607_24959_b300 import workloads as W


def _f64(p):
    return {k: (np.asarray(v, np.float64) if not isinstance(v, int) else v)
            for k, v in p.items()}


def _project_numerically(u, DN, DT, mu):
    """min over z with z_N >= mu |z_T| of 1/2 (u-z)^T diag(DN,DT,DT) (u-z),
    by SLSQP from several starts (a smooth reformulation: z_N >= mu sqrt(|z_T|^2 + tiny))."""
    W_ = np.array([DN, DT, DT])
    scale = np.sqrt(W_)

    def f(x):  # x = sqrt(W) z (better conditioned)
        z = x / scale
        d = u - z
        return 0.5 * float(np.sum(W_ * d * d))

    cons = {"type": "ineq",
            "fun": lambda x: x[0] / scale[0] - mu * np.sqrt((x[1] / scale[1]) ** 2 +
                                                           (x[2] / scale[2]) ** 2 + 1e-300)}
    best = np.inf
    starts = [np.zeros(3), scale * np.array([abs(u[0]) + 1, 0, 0]), scale * u,
              scale * np.array([mu * np.hypot(u[1], u[2]), u[1], u[2]])]
    for x0 in starts:
        res = minimize(f, x0, constraints=[cons], method="SLSQP",
                       options=dict(ftol=1e-15, maxiter=500))
        z = res.x / scale
        if z[0] >= mu * np.hypot(z[1], z[2]) - 1e-9 * (1 + abs(z[0])):
            best = min(best, res.fun)
    return best


def test_cone_cost_matches_numerical_projection():
    rng = np.random.default_rng(3)
    zones = np.zeros(3, int)
    for _ in range(300):
        u = rng.standard_normal(3) * rng.choice([0.1, 1.0, 10.0])
        DN, DT = 10 ** rng.uniform(0, 3, 2)
        mu = rng.uniform(0.1, 1.5)
        z, s, g, h = oracle.ell_cone_one(u, DN, DT, mu)
        zones[z] += 1
        s_num = _project_numerically(u, DN, DT, mu)
        assert abs(s - s_num) <= 1e-6 * max(s_num, 1e-9) + 1e-10, (u, DN, DT, mu, s, s_num)
    assert np.all(zones >= 30), zones


def test_cone_gradient_and_hessian_by_differences():
    rng = np.random.default_rng(4)
    for _ in range(300):
        u = rng.standard_normal(3)
        DN, DT = 10 ** rng.uniform(0, 3, 2)
        mu = rng.uniform(0.1, 1.5)
        z, s, g, h = oracle.ell_cone_one(u, DN, DT, mu)
        hstep = 1e-6
        gnum = np.zeros(3)
        hnum = np.zeros((3, 3))
        same = True
        for k in range(3):
            e = np.zeros(3)
            e[k] = hstep
            zp, sp, gp, _ = oracle.ell_cone_one(u + e, DN, DT, mu)
            zm, sm, gm, _ = oracle.ell_cone_one(u - e, DN, DT, mu)
            same = same and zp == z and zm == z
            gnum[k] = (sp - sm) / (2 * hstep)
            hnum[:, k] = (gp - gm) / (2 * hstep)
        if not same:
            continue
        scale = max(1.0, np.max(np.abs(g)))
        assert np.max(np.abs(gnum - g)) <= 1e-6 * scale
        assert np.max(np.abs(hnum - h)) <= 1e-5 * max(1.0, np.max(np.abs(h)))
        assert np.allclose(h, h.T, atol=1e-12 * max(1.0, np.max(np.abs(h))))
        assert np.min(np.linalg.eigvalsh(0.5 * (h + h.T))) >= -1e-9 * max(1.0, np.max(np.abs(h)))


def test_frictionless_cone_equals_pyramid_on_normal_rows():
    w = W.generate("mu0", 40, 9, 6, seed=21, cond=1e2, cone="elliptic", mu_lo=0.0, mu_hi=0.0)
    for b in range(w.n):
        p = _f64(w.instance(b))
        a, zone, st, it = oracle.ell_solve_one(p["M"], p["J"], p["qfrc"], p["aref"], p["D"],
                                               p["mu"])
        assert st == 0
        nrm = np.arange(0, p["J"].shape[0], 3)
        Jn, arn, Dn = p["J"][nrm], p["aref"][nrm], p["D"][nrm]
        a_p, act, st_p, _ = oracle.solve_one(p["M"], Jn, p["qfrc"], arn, Dn)
        assert st_p == 0
        assert np.max(np.abs(a - a_p)) <= 1e-10 * max(1.0, np.max(np.abs(a_p)))
        adj = oracle.ell_adjoint_one(p["M"], p["J"], p["qfrc"], p["aref"], p["D"], p["mu"], a,
                                     p["g"])
        dq, dr, dJ, _, _ = oracle.adjoint_one(p["M"], Jn, p["qfrc"], arn, Dn, a_p, p["g"])
        assert np.allclose(adj["dqfrc"], dq, rtol=1e-9, atol=1e-12)
        assert np.allclose(adj["daref"][nrm], dr, rtol=1e-9, atol=1e-12)
        assert np.allclose(adj["dJ"][nrm], dJ, rtol=1e-9, atol=1e-12)
        tang = np.setdiff1d(np.arange(p["J"].shape[0]), nrm)
        assert np.all(adj["daref"][tang] == 0) and np.all(adj["dJ"][tang] == 0)


def test_solution_is_stationary_and_minimal():
    rng = np.random.default_rng(5)
    for w in (W.franka_elliptic(8), W.quadruped_elliptic(8)):
        for b in range(w.n):
            p = _f64(w.instance(b))
            args = (p["M"], p["J"], p["qfrc"], p["aref"], p["D"], p["mu"])
            a, zone, st, it = oracle.ell_solve_one(*args)
            assert st == 0
            L0 = oracle.ell_objective_one(*args, a)
            h = 1e-6
            grad = np.array([(oracle.ell_objective_one(*args, a + h * e) -
                              oracle.ell_objective_one(*args, a - h * e)) / (2 * h)
                             for e in np.eye(a.size)])
            scale = max(1.0, np.max(np.abs(p["M"] @ a)), np.max(np.abs(p["qfrc"])))
            assert np.max(np.abs(grad)) <= 1e-6 * scale
            for _ in range(20):
                d = rng.standard_normal(a.size) * 10 ** rng.uniform(-6, -2)
                assert oracle.ell_objective_one(*args, a + d) >= L0 - 1e-12 * max(1.0, abs(L0))


def test_line_search_is_exact_minimiser():
    rng = np.random.default_rng(6)
    w = W.quadruped_elliptic(10)
    for b in range(w.n):
        p = _f64(w.instance(b))
        args = (p["M"], p["J"], p["qfrc"], p["aref"], p["D"], p["mu"])
        a = np.linalg.solve(p["M"], p["qfrc"]) + 0.1 * rng.standard_normal(p["M"].shape[0])
        d = rng.standard_normal(a.size)
        # a descent direction: minus the numerical gradient
        g = np.array([(oracle.ell_objective_one(*args, a + 1e-6 * e) -
                       oracle.ell_objective_one(*args, a - 1e-6 * e)) / 2e-6
                      for e in np.eye(a.size)])
        d = -g if np.linalg.norm(g) > 0 else d
        alpha = oracle.ell_line_search_one(*args, a, d)
        grid = np.linspace(0.0, 3.0 * max(alpha, 1e-3), 3001)
        vals = np.array([oracle.ell_objective_one(*args, a + t * d) for t in grid])
        best = grid[np.argmin(vals)]
        assert abs(alpha - best) <= 2 * (grid[1] - grid[0])
        f0 = oracle.ell_objective_one(*args, a + alpha * d)
        assert f0 <= vals.min() + 1e-12 * max(1.0, abs(f0))


def _loss(p, key, idx, delta):
    q = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in p.items()}
    if key == "M":
        q["M"] = q["M"] + delta * idx
    else:
        q[key].reshape(-1)[idx] += delta
    a, zone, st, _ = oracle.ell_solve_one(q["M"], q["J"], q["qfrc"], q["aref"], q["D"],
                                          q["mu"])
    assert st == 0
    return float(q["g"] @ a), zone


@pytest.mark.parametrize("make", [lambda: W.franka_elliptic(3),
                                  lambda: W.generate("ell-small", 4, 4, 3, seed=23, cond=1e1,
                                                     cone="elliptic", d_lo=1.0, d_hi=3.0)])
def test_adjoint_by_central_differences(make):
    w = make()
    checked = skipped = 0
    for b in range(w.n):
        p = _f64(w.instance(b))
        a, zone, st, _ = oracle.ell_solve_one(p["M"], p["J"], p["qfrc"], p["aref"], p["D"],
                                              p["mu"])
        adj = oracle.ell_adjoint_one(p["M"], p["J"], p["qfrc"], p["aref"], p["D"], p["mu"], a,
                                     p["g"])
        nv, m = p["M"].shape[0], p["J"].shape[0]
        cases = [("qfrc", j, adj["dqfrc"][j]) for j in range(nv)]
        cases += [("aref", i, adj["daref"][i]) for i in range(m)]
        cases += [("J", q, adj["dJ"].ravel()[q]) for q in range(0, m * nv, max(1, m * nv // 40))]
        for j in range(nv):
            for k in range(j + 1):
                E = np.zeros((nv, nv))
                E[j, k] += 1.0
                if j != k:
                    E[k, j] += 1.0
                cases.append(("M", E, float(np.sum(adj["dM"] * E))))
        for c in range(m // 3):
            cases.append(("D", 3 * c, adj["dD"][3 * c]))
            cases.append(("D", 3 * c + 1, adj["dD"][3 * c + 1]))
            cases.append(("mu", 3 * c, adj["dmu"][3 * c]))
        for key, idx, expect in cases:
            ests = {}
            for h in (1e-5, 1e-6):
                hh = h * (max(1.0, abs(p["D"].reshape(-1)[idx])) if key == "D" else 1.0)
                lp, zp = _loss(p, key, idx, +hh)
                lm, zm = _loss(p, key, idx, -hh)
                if not (np.array_equal(zp, zone) and np.array_equal(zm, zone)):
                    ests = None
                    break
                ests[h] = (lp - lm) / (2 * hh)
            if ests is None:
                skipped += 1
                continue
            checked += 1
            scale = max(1e-3, abs(expect))
            assert abs(ests[1e-5] - ests[1e-6]) <= 2e-5 * scale + 1e-8
            assert abs(ests[1e-5] - expect) <= 2e-6 * scale + 1e-8, (key, idx, expect, ests)
    assert checked > 10 * max(skipped, 1)
