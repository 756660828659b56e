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


# FP32 error model of the round cone's adjoint near a zone boundary: the
# gradient, Hessian block and cone-parameter derivatives of a contact whose
# zone margin (relative distance of its u from a zone boundary, as
# _contact_margins measures it) is delta change by about 1/delta per relative
# change of u, and FP32 leaves a with a relative error of about 1e-7, so the
# adjoint of such an instance is resolved to about 1e-7/delta.  Measured
# largest error x delta: 1.0e-8 (nv 96), 7.0e-7 (quadruped), 7e-8 (Franka).
ZONE_ERR = 1e-6


def _check(w, gpu, idx, what, max_over=0.02):
    """Every instance the oracle solves: the GPU solves it, a within 1e-4,
    and each gradient within max(1e-3, ZONE_ERR / delta), delta the
    instance's smallest contact zone margin at the oracle's a.  No instance
    is exempt.  Instances beyond 1e-3 (those with a contact closer than
    about 1e-3 to a zone boundary) are counted: at most max_over of them."""
    ref = oracle.ell_solve_workload(w, idx=idx, threads=8)
    worst = {k: 0.0 for k in ("a",) + KEYS}
    bad, over, worst_ratio = [], 0, 0.0
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
        for k, v in errs.items():
            worst[k] = max(worst[k], v)
        e = max(errs.values())
        if e > parity.G_TOL:
            mg = _contact_margins(w, b, ref["a"][s["a"]])
            delta = float(mg.min()) if mg.size else np.inf
            worst_ratio = max(worst_ratio, e * delta)
            if e > ZONE_ERR / max(delta, 1e-30):
                bad.append((int(b), errs, delta))
                continue
            over += 1
    msg = (f"{what}: worst {worst}, instances beyond 1e-3 {over} (largest error x margin "
           f"{worst_ratio:.2e}), bad {len(bad)} e.g. {bad[:3]}")
    print(msg)
    assert not bad, msg
    assert over <= max_over * len(idx), msg


def test_franka_elliptic(cuda_device):
    w = W.franka_elliptic(n=2048, seed=91)
    gpu = _gpu(w, cuda_device)
    assert np.all(gpu["status"] == 0), np.bincount(gpu["status"])
    _check(w, gpu, np.arange(w.n), "franka elliptic", max_over=0.0)


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


def test_nv96_elliptic_cta(cuda_device):
    """One CTA per instance: nv 96 (the paper's 16-particle point) with 16
    round-cone contacts (48 rows), cond(M) 1e3.  Newton needs 46 steps on
    average here (the FP64 oracle too, two of 256 reach its 100-step cap):
    parity is graded on the instances the oracle solves, and the GPU (allowed
    200 steps) must solve each of those."""
    w = W.generate("nv96_elliptic", 256, 96, 16, seed=97, cond=1e3, cone="elliptic")
    # the GPU may take up to 200 steps: an instance the oracle solves within
    # its 100 can need a few more in FP32, and parity is graded on the
    # oracle's solved instances only
    gpu = _gpu(w, cuda_device, max_iter=200)
    # with 96 DoF against 48 rows the minimiser puts contacts onto the cone's
    # zone boundaries: every instance here has a contact within 1e-4 of one
    # (against 34 % of the quadruped batch), so the count is not capped and
    # the per-instance bound is what holds
    _check(w, gpu, np.arange(w.n), "nv96 elliptic (CTA)", max_over=1.0)


def test_many_contacts_elliptic_cta(cuda_device):
    """One CTA per instance with up to four rows per thread and two contacts
    per thread: 256 round-cone contacts (768 rows) at nv 18 and nv 6, and 341
    (1023 rows, the largest count) at nv 9."""
    for w in (W.generate("c256e-nv18", 48, 18, 256, seed=98, cond=1e3, cone="elliptic"),
              W.generate("c256e-nv6", 48, 6, 256, seed=99, cond=1e2, cone="elliptic"),
              W.generate("c341e-nv9", 24, 9, 341, seed=100, cond=1e2, cone="elliptic")):
        gpu = _gpu(w, cuda_device)
        _check(w, gpu, np.arange(w.n), f"{w.name} (CTA)")


def test_cta_elliptic_on_warp_sized_instances(cuda_device):
    """A batch whose largest instance needs a CTA runs every instance on the
    CTA kernel: the warp-sized ones meet the same parity as on the warp
    kernel."""
    q = W.quadruped_elliptic(n=384, seed=101)
    big = W.generate("big_e", 2, 40, 10, seed=102, cond=1e2, cone="elliptic")
    w = W.pack([q.instance(b) for b in range(q.n)] + [big.instance(b) for b in range(big.n)],
               name="quadruped+big elliptic")
    gpu = _gpu(w, cuda_device)
    _check(w, gpu, np.arange(w.n), "quadruped elliptic on the CTA kernel")


def test_elliptic_cta_edge_cases(cuda_device):
    """CTA-sized round-cone batches with no contacts, frictionless contacts
    (mu = 0), one contact, and a row count that is not a multiple of 3 (a
    shape error for that instance only)."""
    parts = []
    for gen in (lambda: W.generate("c0", 6, 40, 0, seed=103, cond=1e2, cone="elliptic"),
                lambda: W.generate("cmu0", 6, 40, 8, seed=104, cond=1e2, cone="elliptic",
                                   mu_lo=0.0, mu_hi=0.0),
                lambda: W.generate("c1", 6, 64, 1, seed=105, cond=1e2, cone="elliptic")):
        ww = gen()
        parts += [ww.instance(b) for b in range(ww.n)]
    w = W.pack(parts, name="elliptic-cta-edges")
    gpu = _gpu(w, cuda_device)
    # many DoF per contact puts contacts onto zone boundaries (as at nv 96):
    # the per-instance bound holds, the count beyond 1e-3 is not capped
    _check(w, gpu, np.arange(w.n), "elliptic CTA edge cases", max_over=1.0)
    bad = W.pack([dict(M=np.eye(40), J=np.ones((4, 40)), qfrc=np.zeros(40), aref=np.zeros(4),
                       D=np.ones(4), g=np.ones(40), mu=np.ones(4))])
    out = _gpu(bad, cuda_device)
    assert out["status"][0] == 4
