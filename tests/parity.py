"""Shared helpers of the GPU parity tests: run the CUDA path, run the oracle on
the same seeded inputs, compare instance by instance.

Tolerances (per instance, per output array, relative to the oracle's
infinity norm):  a <= 1e-4;  dqfrc, daref, dJ (and dM, dD) <= 1e-3;  active sets
bit-identical on non-degenerate instances.  An instance is degenerate when a
row sits on the cone boundary at the oracle's solution, measured on the scale
that decides its side: a row with |jar_i| < DEG_MARGIN * (sum_k |J_ik a_k| +
|aref_i|), and if it is active also a force |f_i| = D_i |jar_i| <
FORCE_MARGIN * max_k |f_k| (stiff active rows have |jar| = |f| / D far below
|J a| without being near the boundary, and a soft row's small force alone
does not put it there).  There the active set and the adjoint are not
defined (the derivative is local to a fixed contact set), so only a is
compared.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle

A_TOL = 1e-4
G_TOL = 1e-3
DEG_MARGIN = 1e-6
FORCE_MARGIN = 1e-5


def rel(x, y):
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    if y.size == 0:
        return 0.0
    d = np.max(np.abs(x - y))
    return float(d / max(np.max(np.abs(y)), 1e-30))


def run_gpu_fused(batch, w, theta=False, **kw):
    from paper_2607_24959_b300 import solver
    g = torch.from_numpy(np.ascontiguousarray(w.g, np.float32)).to(batch.M.device)
    out = solver.solve_fused(batch, g, theta=theta, **kw)
    torch.cuda.synchronize()
    res = dict(a=out.a.cpu().numpy(), dqfrc=out.dqfrc.cpu().numpy(),
               daref=out.daref.cpu().numpy(), dJ=out.dJ.cpu().numpy(),
               status=out.status.cpu().numpy(), iters=out.iters.cpu().numpy())
    if theta:
        res["dM"] = out.dM.cpu().numpy()
        res["dD"] = out.dD.cpu().numpy()
    return res


def run_gpu_split(batch, w, keep_factor=True, theta=False, **kw):
    from paper_2607_24959_b300 import solver
    g = torch.from_numpy(np.ascontiguousarray(w.g, np.float32)).to(batch.M.device)
    a, st = solver.solve_fwd(batch, keep_factor=keep_factor, **kw)
    grads = solver.solve_adjoint(batch, a, st, g, theta=theta, **kw)
    torch.cuda.synchronize()
    res = dict(a=a.cpu().numpy(), dqfrc=grads[0].cpu().numpy(),
               daref=grads[1].cpu().numpy(), dJ=grads[2].cpu().numpy(),
               status=st.status.cpu().numpy(), iters=st.iters.cpu().numpy(),
               act=st.act.cpu().numpy(), a_lo=st.a_lo.cpu().numpy())
    if theta:
        res["dM"] = grads[3].cpu().numpy()
        res["dD"] = grads[4].cpu().numpy()
    return res


def valid_mask(w):
    """Boolean masks of the real (non-padding) entries of the packed arrays."""
    mv = np.zeros(w.qfrc.size, bool)
    mr = np.zeros(w.aref.size, bool)
    mJ = np.zeros(w.J.size, bool)
    mM = np.zeros(w.M.size, bool)
    for e in w.inst:
        nv, m = int(e["nv"]), int(e["m"])
        mv[e["off_v"]:e["off_v"] + nv] = True
        mr[e["off_r"]:e["off_r"] + m] = True
        mJ[e["off_J"]:e["off_J"] + m * nv] = True
        mM[e["off_M"]:e["off_M"] + nv * nv] = True
    return dict(a=mv, dqfrc=mv, a_lo=mv, daref=mr, act=mr, dJ=mJ, dM=mM, dD=mr)


def valid(w, out, key, masks=None):
    """The real entries of a packed output (or per-instance array as is)."""
    masks = masks or valid_mask(w)
    x = np.asarray(out[key])
    if key in masks:
        return x[:masks[key].size][masks[key]]
    return x[:w.n]


def compare(w, gpu, ref, idx, check_act=True):
    """Per-instance comparison; returns a summary dict (fails nothing).

    Active sets must agree on every row that is not on the boundary (see the
    module docstring).  An instance whose active sets agree on all rows gets
    the full check (a and every gradient); one whose sets differ only on
    boundary rows (a legitimate flip: the derivative is not defined there)
    gets the a check and is counted in ``flipped``.
    """
    theta = "dM" in gpu and "dM" in ref
    worst = dict(a=0.0, dqfrc=0.0, daref=0.0, dJ=0.0)
    if theta:
        worst.update(dM=0.0, dD=0.0)
    bad = []
    degenerate = 0
    flipped = 0
    act_mismatch = []
    for b in idx:
        e = w.inst[b]
        nv, m = int(e["nv"]), int(e["m"])
        ov, orr, oJ = int(e["off_v"]), int(e["off_r"]), int(e["off_J"])
        oM = int(e["off_M"])
        if ref["status"][b] != 0:
            continue
        p = w.instance(b)
        a_ref = ref["a"][ov:ov + nv]
        jar = p["J"].astype(np.float64) @ a_ref - p["aref"]
        scale = np.abs(p["J"].astype(np.float64)) @ np.abs(a_ref) + np.abs(p["aref"])
        f = p["D"].astype(np.float64) * np.minimum(jar, 0.0)
        fmax = np.max(np.abs(f)) if m else 0.0
        near = ((np.abs(jar) < DEG_MARGIN * scale)
                & ((jar >= 0) | (np.abs(f) < FORCE_MARGIN * fmax))) if m else np.zeros(0, bool)
        degenerate += bool(np.any(near))
        ea = rel(gpu["a"][ov:ov + nv], a_ref)
        worst["a"] = max(worst["a"], ea)
        same = True
        if check_act and m:
            act_ref = ref["act"][orr:orr + m].astype(bool)
            if "act" in gpu:
                act_gpu = gpu["act"][orr:orr + m].astype(bool)
            else:
                # daref is zero exactly on inactive rows (an active row with
                # J w = 0 exactly does not occur with continuous random data)
                act_gpu = gpu["daref"][orr:orr + m] != 0
            diff = act_gpu != act_ref
            if np.any(diff & ~near):
                act_mismatch.append(int(b))
                bad.append((int(b), dict(a=ea, act="mismatch off the boundary"),
                            int(gpu["status"][b]), int(gpu["iters"][b])))
                continue
            same = not np.any(diff)
        if not same:
            flipped += 1
            if ea > A_TOL or gpu["status"][b] != 0:
                bad.append((int(b), dict(a=ea), int(gpu["status"][b]), int(gpu["iters"][b])))
            continue
        errs = dict(
            a=ea,
            dqfrc=rel(gpu["dqfrc"][ov:ov + nv], ref["dqfrc"][ov:ov + nv]),
            daref=rel(gpu["daref"][orr:orr + m], ref["daref"][orr:orr + m]) if m else 0.0,
            dJ=rel(gpu["dJ"][oJ:oJ + m * nv], ref["dJ"][oJ:oJ + m * nv]) if m else 0.0,
        )
        if theta:
            errs["dM"] = rel(gpu["dM"][oM:oM + nv * nv], ref["dM"][oM:oM + nv * nv])
            errs["dD"] = rel(gpu["dD"][orr:orr + m], ref["dD"][orr:orr + m]) if m else 0.0
        for k, v in errs.items():
            worst[k] = max(worst[k], v)
        ok = (errs["a"] <= A_TOL and all(v <= G_TOL for k, v in errs.items() if k != "a")
              and gpu["status"][b] == 0)
        if not ok:
            bad.append((int(b), errs, int(gpu["status"][b]), int(gpu["iters"][b])))
    return dict(worst=worst, bad=bad, degenerate=degenerate, flipped=flipped,
                act_mismatch=act_mismatch, checked=len(idx))
