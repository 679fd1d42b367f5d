"""The multi-rank path on CPU (gloo, world size 2): every rank runs its own
share of independent replicas/groups with its own seeds and no exchange on the
data path; the only collective is the max of the per-rank times.  Results of a
rank equal a single-process run with the same seeds (placement independence of
the counter-based stream)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as tmp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import core
    Ls, betas, seeds = bench.workload(rank)
    g = int(np.argmin(Ls))  # this rank's smallest group, 2 steps on the oracle
    L = int(Ls[g])
    s0 = core.lattice_init(L, 32, seeds[g], core.MODE_MULTISPIN, 0)
    s1, _ = core.lattice_run(s0, 1.0, 1.0, 0.0, betas[32 * g:32 * g + 32], seeds[g], 0, 2,
                             core.MODE_MULTISPIN)
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    q.put((rank, list(seeds), g, int(s1.sum()), float(t.item())))
    dist.destroy_process_group()


def test_two_rank_sharding_gloo():
    pytest.importorskip("torch.distributed")
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, seeds0, g0, sum0, t0), (r1, seeds1, g1, sum1, t1) = res
    assert not set(seeds0) & set(seeds1)  # disjoint streams per rank
    assert t0 == t1 == 2.0                # max over ranks
    # rank 1's result equals a single-process run with rank 1's seeds
    import bench
    from oracle import core
    Ls, betas, seeds = bench.workload(1)
    L = int(Ls[g1])
    s0 = core.lattice_init(L, 32, seeds[g1], core.MODE_MULTISPIN, 0)
    s1, _ = core.lattice_run(s0, 1.0, 1.0, 0.0, betas[32 * g1:32 * g1 + 32], seeds[g1], 0, 2,
                             core.MODE_MULTISPIN)
    assert int(s1.sum()) == sum1
