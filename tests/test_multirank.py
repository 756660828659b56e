"""The benchmark's N > 1 path on CPU with the gloo backend (world size 2):
every rank owns a disjoint, independently seeded shard of instances (weak
scaling, no data exchange); the only collectives are the barrier and the MAX
reduction of the timed region.  The per-rank solves run through the oracle
here because this machine has no GPU."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    import bench
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = bench.make_workload("tiny", rank, n=64)
    out = oracle.solve_workload(w)
    local_ms = 10.0 + 5.0 * rank                     # a stand-in timing
    t = torch.tensor([local_ms], dtype=torch.float64)
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q.put((rank, float(t.item()), int(w.params["seed"]), out["a"].copy(),
           int(np.sum(out["status"] == 0))))
    dist.destroy_process_group()


def test_two_rank_weak_scaling_shards():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, s0, a0, ok0), (r1, t1, s1, a1, ok1) = res
    assert t0 == t1 == 15.0                 # max over ranks
    assert s0 != s1                         # independent shards
    assert ok0 == ok1 == 64
    assert not np.allclose(a0, a1)
    import bench
    import oracle
    w1 = bench.make_workload("tiny", 1, n=64)   # a rank's shard alone
    assert np.array_equal(oracle.solve_workload(w1)["a"], a1)
