"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs, instance by instance (tolerances in tests/parity.py).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_24959_b300 import solver, workloads as W
from tests import parity

pytestmark = pytest.mark.gpu


def _check(w, gpu, idx, what, max_flipped_frac=0.02):
    ref = oracle.solve_workload(w, idx=idx, threads=8)
    res = parity.compare(w, gpu, ref, idx)
    msg = (f"{what}: worst {res['worst']}, instances with a boundary row "
           f"{res['degenerate']}/{res['checked']}, boundary flips {res['flipped']}, "
           f"failing {len(res['bad'])} e.g. {res['bad'][:3]}, "
           f"active-set mismatches {res['act_mismatch'][:5]}")
    print(msg)
    assert not res["bad"], msg
    assert res["flipped"] <= max_flipped_frac * max(res["checked"], 1), msg
    return res


def test_tiny_full_fused_and_split(cuda_device):
    w = W.tiny()
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    idx = np.arange(w.n)
    _check(w, parity.run_gpu_fused(batch, w), idx, "tiny fused")
    _check(w, parity.run_gpu_split(batch, w), idx, "tiny split")


def test_franka_full(cuda_device):
    w = W.franka()
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    _check(w, parity.run_gpu_fused(batch, w), np.arange(w.n), "franka fused")


def test_quadruped_small_all_instances(cuda_device):
    # several tiles of warps and a ragged tail, every instance checked
    w = W.quadruped(n=1000)
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    _check(w, parity.run_gpu_fused(batch, w), np.arange(w.n), "quadruped-1000 fused")
    _check(w, parity.run_gpu_split(batch, w), np.arange(w.n), "quadruped-1000 split")


def test_quadruped_full_size_sampled(cuda_device):
    """The benchmark's workload (32768 ragged instances) in the benchmark's
    launch configuration (fused, cost-ordered claims); a sample of 2048
    instances is checked against the oracle."""
    w = W.quadruped()
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    order = torch.from_numpy(solver.cost_order(w.inst)).to(cuda_device)
    gpu = parity.run_gpu_fused(batch, w, order=order)
    assert np.all(gpu["status"] == 0), np.bincount(gpu["status"])
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(w.n, 2048, replace=False))
    _check(w, gpu, idx, "quadruped-32768 fused (sampled)")


@pytest.mark.parametrize("name,extra_steps", [("quadruped", 1.25), ("franka", 0.75), ("nv96", 3.0)])
def test_newton_steps_and_accuracy_against_the_oracle(cuda_device, name, extra_steps):
    """The GPU takes the oracle's Newton steps plus the refinement steps the
    FP32 contract costs (the oracle ends on exact termination after the step
    that keeps the active set; in FP32 that step leaves a with the error of
    an FP32 solve, removed by one refinement step, two to three at cond(M)
    1e4), and returns a near FP32 resolution and gradients near 1e-5: far
    inside the parity tolerances, which a looser stop rule would still meet."""
    gen = {"quadruped": lambda: W.quadruped(n=2048, seed=81),
           "franka": lambda: W.franka(n=2048, seed=82),
           "nv96": lambda: W.nv96(n=192, seed=83)}[name]
    w = gen()
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    gpu = parity.run_gpu_fused(batch, w)
    ref = oracle.solve_workload(w, threads=8)
    ok = (gpu["status"][:w.n] == 0) & (ref["status"][:w.n] == 0)
    assert ok.mean() > 0.99
    g_it = gpu["iters"][:w.n][ok].mean()
    o_it = ref["iters"][:w.n][ok].mean()
    print(f"{name}: GPU {g_it:.2f} Newton steps per solve, oracle {o_it:.2f}")
    assert g_it <= o_it + extra_steps, (g_it, o_it)
    worst_a = worst_g = 0.0
    for b in np.flatnonzero(ok):
        e = w.inst[b]
        nv, m = int(e["nv"]), int(e["m"])
        ov, orr, oJ = int(e["off_v"]), int(e["off_r"]), int(e["off_J"])
        worst_a = max(worst_a, parity.rel(gpu["a"][ov:ov + nv], ref["a"][ov:ov + nv]))
        for k, sl in (("dqfrc", slice(ov, ov + nv)), ("daref", slice(orr, orr + m)),
                      ("dJ", slice(oJ, oJ + m * nv))):
            worst_g = max(worst_g, parity.rel(gpu[k][sl], ref[k][sl]))
    print(f"{name}: worst relative error a {worst_a:.2e}, gradients {worst_g:.2e}")
    assert worst_a <= 5e-6 and worst_g <= 2e-4, (worst_a, worst_g)


def test_fused_equals_split_bitwise(cuda_device):
    """The fused kernel and the split forward + adjoint with the kept factor
    share the forward and the adjoint solve bit for bit (a, status, iters, w =
    dqfrc and lambda = daref).  The forces f in dJ = -(f w^T + lambda a^T)
    differ in their last bits: a fused solve that stops after a refinement
    step advances f along that step, the split adjoint re-evaluates f at the
    returned a.  Recompute mode rebuilds the Newton matrix of the returned
    active set from M, where the forward formed it by row updates, so its
    gradients agree to the refinement's accuracy."""
    w = W.quadruped(n=700, seed=77)
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    f = parity.run_gpu_fused(batch, w)
    s1 = parity.run_gpu_split(batch, w, keep_factor=True)
    s0 = parity.run_gpu_split(batch, w, keep_factor=False)
    masks = parity.valid_mask(w)
    for k in ("a", "dqfrc", "daref", "status", "iters"):
        assert np.array_equal(parity.valid(w, f, k, masks), parity.valid(w, s1, k, masks)), k
    x = parity.valid(w, f, "dJ", masks).astype(np.float64)
    y = parity.valid(w, s1, "dJ", masks).astype(np.float64)
    assert np.max(np.abs(x - y)) <= 1e-6 * max(np.max(np.abs(y)), 1e-30)
    for k in ("a", "status", "iters"):
        assert np.array_equal(parity.valid(w, s0, k, masks), parity.valid(w, s1, k, masks)), k
    for k in ("dqfrc", "daref", "dJ"):
        x = parity.valid(w, s0, k, masks).astype(np.float64)
        y = parity.valid(w, s1, k, masks).astype(np.float64)
        assert np.max(np.abs(x - y)) <= 1e-4 * max(np.max(np.abs(y)), 1e-30), k


def test_launch_shape_and_order_do_not_change_results(cuda_device):
    w = W.quadruped(n=900, seed=5)
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    base = parity.run_gpu_fused(batch, w)
    masks = parity.valid_mask(w)
    order = torch.from_numpy(solver.cost_order(w.inst)).to(cuda_device)
    rev = torch.flip(torch.arange(w.n, dtype=torch.int32, device=cuda_device), [0])
    for kw in (dict(order=order), dict(order=rev), dict(warps_per_block=1),
               dict(warps_per_block=8)):
        o = parity.run_gpu_fused(batch, w, **kw)
        for k in ("a", "dqfrc", "daref", "dJ", "status", "iters"):
            assert np.array_equal(parity.valid(w, o, k, masks),
                                  parity.valid(w, base, k, masks)), (kw, k)


def test_plan_matches_single_kernel_bitwise(cuda_device):
    w = W.quadruped(n=3000, seed=31)
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    g = torch.from_numpy(w.g).to(cuda_device)
    single = parity.run_gpu_fused(batch, w)
    plan = solver.FusedPlan(batch, g, autotune=True, graph=True)
    info = plan.describe()
    assert info["graph"] and info["kernels"] >= 3, info     # MT 1, 2, 4 buckets
    assert sum(b["instances"] for b in info["buckets"]) == w.n
    for _ in range(2):                                       # replays are repeatable
        out = plan.launch()
        torch.cuda.synchronize()
        got = dict(a=out.a.cpu().numpy(), dqfrc=out.dqfrc.cpu().numpy(),
                   daref=out.daref.cpu().numpy(), dJ=out.dJ.cpu().numpy(),
                   status=out.status.cpu().numpy(), iters=out.iters.cpu().numpy())
        masks = parity.valid_mask(w)
        for k in ("a", "dqfrc", "daref", "dJ", "status", "iters"):
            assert np.array_equal(parity.valid(w, got, k, masks),
                                  parity.valid(w, single, k, masks)), k
    plan.close()


def _mixed_workload():
    parts = []
    for gen, n in ((lambda: W.tiny(n=200, seed=3), 200),
                   (lambda: W.franka(n=200, seed=4), 200),
                   (lambda: W.quadruped(n=200, seed=5), 200),
                   (lambda: W.generate("nv32", 60, 32, 64, seed=6, cond=1e3), 60),
                   (lambda: W.generate("nv5", 60, 5, 7, seed=7, cond=1e2), 60),
                   (lambda: W.generate("nv1", 40, 1, 3, seed=8, cond=1.0), 40)):
        w = gen()
        parts += [w.instance(b) for b in range(n)]
    rng = np.random.default_rng(0)
    parts = [parts[i] for i in rng.permutation(len(parts))]
    return W.pack(parts, name="mixed")


def test_mixed_nv_plan_parity(cuda_device):
    w = _mixed_workload()
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    g = torch.from_numpy(w.g).to(cuda_device)
    plan = solver.FusedPlan(batch, g, autotune=False, graph=True)
    assert plan.describe()["kernels"] >= 4
    out = plan.launch()
    torch.cuda.synchronize()
    gpu = dict(a=out.a.cpu().numpy(), dqfrc=out.dqfrc.cpu().numpy(),
               daref=out.daref.cpu().numpy(), dJ=out.dJ.cpu().numpy(),
               status=out.status.cpu().numpy(), iters=out.iters.cpu().numpy())
    _check(w, gpu, np.arange(w.n), "mixed nv plan")
    plan.close()


def test_edge_cases(cuda_device):
    # nc = 0 everywhere (closed form), nv = 1, the largest supported sizes,
    # offsets that are not multiples of 4 (no 16-byte loads)
    cases = [W.generate("nc0", 100, 18, 0, seed=9),
             W.generate("nv1", 50, 1, 2, seed=10, cond=1.0),
             W.generate("max", 40, 32, 64, seed=11, cond=1e3)]
    odd = W.generate("odd", 30, 7, 3, seed=12, cond=1e2)
    parts = [odd.instance(b) for b in range(odd.n)]
    inst, tM, tJ, tv, tr = W.layout([7] * 30, [12] * 30)
    # re-pack without alignment padding
    M = np.concatenate([p["M"].ravel() for p in parts])
    J = np.concatenate([p["J"].ravel() for p in parts])
    q = np.concatenate([p["qfrc"] for p in parts])
    g = np.concatenate([p["g"] for p in parts])
    ar = np.concatenate([p["aref"] for p in parts])
    D = np.concatenate([p["D"] for p in parts])
    inst["off_M"] = np.arange(30) * 49
    inst["off_J"] = np.arange(30) * 84
    inst["off_v"] = np.arange(30) * 7
    inst["off_r"] = np.arange(30) * 12
    cases.append(W.Workload("unaligned", inst, M, J, q, ar, D, g, {}))
    for w in cases:
        batch = solver.DeviceBatch.from_workload(w, cuda_device)
        _check(w, parity.run_gpu_fused(batch, w), np.arange(w.n), w.name)
        _check(w, parity.run_gpu_split(batch, w), np.arange(w.n), w.name + " split")


def _pack_unaligned(parts, name):
    """Pack instances back to back, with a one-float gap before every third
    block, so that no block is 16-byte aligned by construction."""
    nvs = [int(p["M"].shape[0]) for p in parts]
    ms = [int(p["J"].size // nv) for p, nv in zip(parts, nvs)]
    inst, _, _, _, _ = W.layout(nvs, ms)
    arrays = {k: [] for k in ("M", "J", "qfrc", "aref", "D", "g")}
    ends = {"M": 0, "J": 0, "v": 0, "r": 0}
    for b, p in enumerate(parts):
        gap = 1 if b % 3 == 1 else 0
        for key, names in (("M", ("M",)), ("J", ("J",)), ("v", ("qfrc", "g")),
                           ("r", ("aref", "D"))):
            inst["off_" + key][b] = ends[key] + gap
            for k in names:
                arrays[k].append(np.zeros(gap, np.float32))
                arrays[k].append(np.ravel(p[k]).astype(np.float32))
            ends[key] += gap + np.ravel(p[names[0]]).size
    cat = {k: np.concatenate(v) for k, v in arrays.items()}
    return W.Workload(name, inst, cat["M"], cat["J"], cat["qfrc"], cat["aref"], cat["D"],
                      cat["g"], {})


def test_padded_instances_in_the_asynchronously_staged_kernels(cuda_device):
    # nv below the kernel's NV (M padded with identity rows, J with zero
    # columns, written by plain stores beside the asynchronous copies) in the
    # kernels that stage by 4-byte cp.async (NV >= 16, or more than 64 rows),
    # at every rows-per-lane count, packed with no block aligned
    parts = []
    for nv, nc, seed in ((13, 30, 21), (11, 24, 22), (17, 12, 23), (13, 8, 24), (25, 12, 25),
                         (7, 20, 26)):
        w = W.generate(f"pad{nv}", 20, nv, nc, seed=seed, cond=1e3)
        parts += [w.instance(b) for b in range(w.n)]
    rng = np.random.default_rng(27)
    w = _pack_unaligned([parts[i] for i in rng.permutation(len(parts))], "padded-async")
    assert np.any(w.inst["off_J"] % 4 != 0) and np.any(w.inst["off_M"] % 4 != 0)
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    _check(w, parity.run_gpu_fused(batch, w), np.arange(w.n), w.name)
    _check(w, parity.run_gpu_split(batch, w), np.arange(w.n), w.name + " split")
    g = torch.from_numpy(w.g).to(cuda_device)
    plan = solver.FusedPlan(batch, g, autotune=False, graph=True)
    out = plan.launch()
    torch.cuda.synchronize()
    got = dict(a=out.a.cpu().numpy(), dqfrc=out.dqfrc.cpu().numpy(),
               daref=out.daref.cpu().numpy(), dJ=out.dJ.cpu().numpy(),
               status=out.status.cpu().numpy(), iters=out.iters.cpu().numpy())
    plan.close()
    _check(w, got, np.arange(w.n), w.name + " plan")


def test_cuda_path_matches_exact_golden_solutions(cuda_device):
    # the stored exact minimisers and adjoints (exact rational arithmetic,
    # tests/golden/make_golden.py), independent of the oracle
    from tests.test_golden import load_cases
    cases = load_cases()
    parts = [dict(M=np.asarray(c["M"], np.float32),
                  J=np.asarray(c["J"], np.float32).reshape(c["m"], c["nv"]),
                  qfrc=np.asarray(c["qfrc"], np.float32), aref=np.asarray(c["aref"], np.float32),
                  D=np.asarray(c["D"], np.float32), g=np.asarray(c["g"], np.float32))
             for c in cases]
    w = W.pack(parts, name="golden")
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    for label, got in (("fused", parity.run_gpu_fused(batch, w)),
                       ("split", parity.run_gpu_split(batch, w))):
        for b, c in enumerate(cases):
            e = w.inst[b]
            nv, m = int(e["nv"]), int(e["m"])
            ov, orr, oJ = int(e["off_v"]), int(e["off_r"]), int(e["off_J"])
            assert got["status"][b] == 0, (label, c["name"])
            assert parity.rel(got["a"][ov:ov + nv], c["a"]) <= parity.A_TOL, (label, c["name"])
            assert parity.rel(got["dqfrc"][ov:ov + nv], c["dqfrc"]) <= parity.G_TOL
            dr = got["daref"][orr:orr + m]
            assert parity.rel(dr, c["daref"]) <= parity.G_TOL, (label, c["name"])
            assert ((dr != 0).astype(int).tolist() == c["active"]), (label, c["name"])
            assert parity.rel(got["dJ"][oJ:oJ + m * nv], np.ravel(c["dJ"])) <= parity.G_TOL


def test_max_rows_per_instance(cuda_device):
    w = W.generate("m256", 64, 18, 64, seed=13, cond=1e3)     # m = 256 rows
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    _check(w, parity.run_gpu_fused(batch, w), np.arange(w.n), "m=256")


def test_empty_batch_and_bad_shapes(cuda_device):
    w = W.quadruped(n=10, seed=14)
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    empty = solver.DeviceBatch(batch.inst, batch.M, batch.J, batch.qfrc, batch.aref,
                               batch.D, 0, 1, 0, w.inst[:0])
    g = torch.zeros(4, device=cuda_device)
    solver.solve_fused(empty, g)                          # no-op, no error
    # an instance larger than the batch bound is flagged, the others solve
    inst = w.inst.copy()
    inst["m"][3] = 200                                    # > m_max of the batch
    bad = solver.DeviceBatch(torch.from_numpy(inst.view(np.uint8)).to(cuda_device),
                             batch.M, batch.J, batch.qfrc, batch.aref, batch.D,
                             w.n, 18, 128, inst)
    out = solver.solve_fused(bad, torch.from_numpy(w.g).to(cuda_device))
    torch.cuda.synchronize()
    st = out.status.cpu().numpy()[:w.n]
    assert st[3] == 4 and np.all(np.delete(st, 3) == 0), st


def test_nonfinite_input_is_a_status(cuda_device):
    w = W.quadruped(n=20, seed=15)
    w.qfrc[w.inst["off_v"][5]] = np.nan
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    out = solver.solve_fused(batch, torch.from_numpy(w.g).to(cuda_device))
    torch.cuda.synchronize()
    st = out.status.cpu().numpy()[:w.n]
    assert st[5] == 3 and np.all(np.delete(st, 5) == 0), st


def test_iteration_cap_status(cuda_device):
    w = W.quadruped(n=200, seed=16)
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    out = solver.solve_fused(batch, torch.from_numpy(w.g).to(cuda_device), max_iter=1)
    torch.cuda.synchronize()
    st = out.status.cpu().numpy()[:w.n]
    it = out.iters.cpu().numpy()[:w.n]
    assert np.all(it <= 1) and np.any(st == 1) and set(np.unique(st)) <= {0, 1}


def test_host_pipeline_matches_device_path(cuda_device):
    w = W.quadruped(n=3000, seed=71)
    pipe = solver.HostPipeline(w, chunks=5, device=cuda_device)
    for _ in range(2):
        pipe.step()
    torch.cuda.synchronize()
    got = {k: v.numpy() for k, v in pipe.h_out.items()}
    pipe.close()
    batch = solver.DeviceBatch.from_workload(w, cuda_device)
    ref = parity.run_gpu_fused(batch, w)
    masks = parity.valid_mask(w)
    for k in ("a", "dqfrc", "daref", "dJ", "status", "iters"):
        assert np.array_equal(parity.valid(w, got, k, masks), parity.valid(w, ref, k, masks)), k
