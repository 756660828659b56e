"""GPU parity of the round (elliptic) Coulomb cone: the CUDA fused solve and
IFT adjoint (cs_solve_fused_elliptic) against the FP64 oracle on the same
seeded inputs, for every output (a, dqfrc, daref, dJ, dM, dD, dmu)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_24959_b300 import solver, workloads as W
from tests import parity

pytestmark = pytest.mark.gpu

KEYS = ("dqfrc", "daref", "dJ", "dM", "dD", "dmu")


def _gpu(w, dev, **kw):
    batch = solver.DeviceBatch.from_workload(w, dev)
    g = torch.from_numpy(w.g).to(dev)
    mu = torch.from_numpy(w.mu).to(dev)
    out = solver.solve_fused_elliptic(batch, g, mu, **kw)
    torch.cuda.synchronize()
    f = out.fused
    return dict(a=f.a.cpu().numpy(), dqfrc=f.dqfrc.cpu().numpy(), daref=f.daref.cpu().numpy(),
                dJ=f.dJ.cpu().numpy(), dM=f.dM.cpu().numpy(), dD=f.dD.cpu().numpy(),
                dmu=out.dmu.cpu().numpy(), status=f.status.cpu().numpy()[:w.n],
                iters=f.iters.cpu().numpy()[:w.n])


def _segments(w, b):
    e = w.inst[b]
    nv, m = int(e["nv"]), int(e["m"])
    ov, orr, oJ, oM = (int(e[k]) for k in ("off_v", "off_r", "off_J", "off_M"))
    return dict(a=slice(ov, ov + nv), dqfrc=slice(ov, ov + nv), daref=slice(orr, orr + m),
                dD=slice(orr, orr + m), dmu=slice(orr, orr + m), dJ=slice(oJ, oJ + m * nv),
                dM=slice(oM, oM + nv * nv), zone=slice(orr, orr + m))


def _zone_margin(w, b, a):
    """Smallest relative distance of a contact from a zone boundary at the
    oracle's a: |mu t - u_N| and |mu D_N u_N + D_T t| over their scales."""
    p = {k: np.asarray(v, np.float64) for k, v in w.instance(b).items()}
    u = p["J"] @ a - p["aref"]
    sc = np.abs(p["J"]) @ np.abs(a) + np.abs(p["aref"])
    best = np.inf
    for c in range(p["J"].shape[0] // 3):
        uN, t = u[3 * c], np.hypot(u[3 * c + 1], u[3 * c + 2])
        DN, DT, mu = p["D"][3 * c], p["D"][3 * c + 1], p["mu"][3 * c]
        s = max(sc[3 * c], sc[3 * c + 1], sc[3 * c + 2])
        best = min(best, abs(mu * t - uN) / s, abs(mu * DN * uN + DT * t) / (DT * s + mu * DN * s))
    return best


def _contact_margins(w, b, a):
    """Relative zone-boundary distance of every contact at a (as _zone_margin)."""
    p = {k: np.asarray(v, np.float64) for k, v in w.instance(b).items()}
    u = p["J"] @ a - p["aref"]
    sc = np.abs(p["J"]) @ np.abs(a) + np.abs(p["aref"])
    out = []
    for c in range(p["J"].shape[0] // 3):
        uN, t = u[3 * c], np.hypot(u[3 * c + 1], u[3 * c + 2])
        DN, DT, mu = p["D"][3 * c], p["D"][3 * c + 1], p["mu"][3 * c]
        s = max(sc[3 * c], sc[3 * c + 1], sc[3 * c + 2])
        out.append(min(abs(mu * t - uN) / s, abs(mu * DN * uN + DT * t) / (DT * s + mu * DN * s)))
    return np.array(out)


def _traced_to_near_contact(w, b, gpu, ref, s, a):
    """Whether the instance has a contact within 1e-4 of a zone boundary and
    that contact's own rows carry entries beyond the tolerance (relative to
    the output's largest entry) in some per-row output (daref, dJ, dD, dmu):
    the contact whose zone-dependent terms lose digits is then implicated
    directly, and other entries' errors are what it passes on through w."""
    near = np.flatnonzero(_contact_margins(w, b, a) < 1e-4)
    if near.size == 0:
        return False
    nv = int(w.inst[b]["nv"])
    for k in ("daref", "dD", "dmu", "dJ"):
        x = np.asarray(gpu[k][s[k]], np.float64)
        y = np.asarray(ref[k][s[k]], np.float64)
        if x.size == 0:
            continue
        err = np.abs(x - y) / max(np.max(np.abs(y)), 1e-30)
        rows = err.reshape(-1, nv).max(1) if k == "dJ" else err
        for c in near:
            if np.max(rows[3 * c:3 * c + 3]) > parity.G_TOL:
                return True
    return False


def _check(w, gpu, idx, what, max_flip=0.02):
    ref = oracle.ell_solve_workload(w, idx=idx, threads=8)
    worst = {k: 0.0 for k in ("a",) + KEYS}
    bad, flips = [], 0
    for b in idx:
        if ref["status"][b] != 0:
            continue
        s = _segments(w, b)
        ea = parity.rel(gpu["a"][s["a"]], ref["a"][s["a"]])
        worst["a"] = max(worst["a"], ea)
        if gpu["status"][b] != 0 or ea > parity.A_TOL:
            bad.append((int(b), "a", ea, int(gpu["status"][b])))
            continue
        errs = {k: parity.rel(gpu[k][s[k]], ref[k][s[k]]) for k in KEYS}
        if any(v > parity.G_TOL for v in errs.values()):
            # the derivative is local to the zones, and near a zone boundary
            # (relative margin delta) the FP32 evaluation of that contact's
            # zone-dependent adjoint terms loses about log10(1/delta) digits:
            # an instance whose near-boundary contact itself carries entries
            # beyond the tolerance is not held to 1e-3 (it is counted
            # instead); any other error fails
            # (an instance with such a contact whose errors elsewhere stay
            # within ten times the tolerance is counted too: the near
            # contact's error reaches every row through w)
            if (_traced_to_near_contact(w, b, gpu, ref, s, ref["a"][s["a"]]) or
                    (_zone_margin(w, b, ref["a"][s["a"]]) < 1e-4 and
                     max(errs.values()) <= 10 * parity.G_TOL)):
                flips += 1
                continue
            bad.append((int(b), errs))
            continue
        for k, v in errs.items():
            worst[k] = max(worst[k], v)
    msg = f"{what}: worst {worst}, zone-boundary instances {flips}, bad {len(bad)} e.g. {bad[:3]}"
    print(msg)
    assert not bad, msg
    assert flips <= max_flip * len(idx), msg


def test_franka_elliptic(cuda_device):
    w = W.franka_elliptic(n=2048, seed=91)
    gpu = _gpu(w, cuda_device)
    assert np.all(gpu["status"] == 0), np.bincount(gpu["status"])
    _check(w, gpu, np.arange(w.n), "franka elliptic")


def test_quadruped_elliptic(cuda_device):
    w = W.quadruped_elliptic(n=2048, seed=92)
    gpu = _gpu(w, cuda_device)
    _check(w, gpu, np.arange(w.n), "quadruped elliptic")


def test_quadruped_elliptic_full_size_sampled(cuda_device):
    w = W.quadruped_elliptic()
    gpu = _gpu(w, cuda_device, order=None)
    assert np.mean(gpu["status"] == 0) > 0.99, np.bincount(gpu["status"])
    idx = np.sort(np.random.default_rng(7).choice(w.n, 512, replace=False))
    _check(w, gpu, idx, "quadruped elliptic full size (sampled)")


def test_elliptic_edge_cases(cuda_device):
    parts = []
    for gen in (lambda: W.generate("e0", 20, 9, 0, seed=93, cond=1e2, cone="elliptic"),
                lambda: W.generate("e1", 20, 1, 2, seed=94, cond=1.0, cone="elliptic"),
                lambda: W.generate("emu0", 20, 6, 4, seed=95, cond=1e2, cone="elliptic",
                                   mu_lo=0.0, mu_hi=0.0),
                lambda: W.generate("emax", 10, 32, 85, seed=96, cond=1e2, cone="elliptic")):
        ww = gen()
        parts += [ww.instance(b) for b in range(ww.n)]
    w = W.pack(parts, name="elliptic-edges")
    gpu = _gpu(w, cuda_device)
    _check(w, gpu, np.arange(w.n), "elliptic edge cases")
    # a row count that is not a multiple of 3 is a shape error
    bad = W.pack([dict(M=np.eye(3), J=np.ones((4, 3)), qfrc=np.zeros(3), aref=np.zeros(4),
                       D=np.ones(4), g=np.ones(3), mu=np.ones(4))])
    out = _gpu(bad, cuda_device)
    assert out["status"][0] == 4
