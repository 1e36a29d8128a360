"""The N > 1 host path with two gloo ranks on the CPU: per-rank shards are
disjoint and deterministic, and the timing / step-count reductions give the
max and the sum over ranks (what bench.py reports under torchrun)."""
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
    import torch.distributed as dist

    from paper_2511_03655_gb300 import dist as pd
    from paper_2511_03655_gb300 import workloads
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = pd.world()
    wl = workloads.kepler_ensemble(batch=256, periods=1, seed_id=pd.shard_seed(2, r))
    pd.barrier()
    t_max = pd.reduce_max(1.0 + r)          # per-rank "time"
    steps = pd.reduce_sum(float(wl["nsteps"].sum()))
    q.put((r, w, lr, wl["e"][:8].tolist(), t_max, steps, float(wl["nsteps"].sum())))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, e0, t0, s0, n0), (r1, w1, l1, e1, t1, s1, n1) = res
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert e0 != e1                                  # disjoint shards
    from paper_2511_03655_gb300 import workloads
    assert np.allclose(e0, workloads.kepler_ensemble(batch=256, periods=1)["e"][:8])  # rank 0 = standard
    assert t0 == t1 == 2.0                           # max over ranks
    assert s0 == s1 == n0 + n1                       # sum over ranks
