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


def _agg_worker(rank, world, port, q, planted):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    Ls, _, seeds = bench.workload(rank)
    steps = 20
    ms = 10.0 * (rank + 1)  # a fake per-rank duration: rank 1 is the slow one
    upd = bench.updates_per_step(Ls) * steps
    if planted:  # a plausible mistake: every rank also counts the others' updates
        upd *= world
    value, ms_max = bench.aggregate(upd, ms, world)
    q.put((rank, len(seeds), value, ms_max))
    dist.destroy_process_group()


def _run_agg(planted):
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_agg_worker, args=(r, 2, port, q, planted)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def _check_agg(res):
    import bench
    # the job: every rank's own groups (weak scaling), summed, over the slowest rank
    expected = sum(bench.updates_per_step(bench.workload(r)[0]) * 20 for r in range(2)) / 0.020
    for rank, ngroups, value, ms_max in res:
        assert ngroups == bench.GROUPS
        assert ms_max == 20.0
        assert abs(value - expected) <= 1e-9 * expected, (value, expected)


def test_bench_rank_aggregation_gloo():
    """bench.py's rank path (bench.aggregate over gloo, world size 2) with fake per-rank
    times: value = the updates of both ranks' groups over the slower rank's time, the
    same on every rank; a planted double count of the updates is rejected."""
    pytest.importorskip("torch.distributed")
    _check_agg(_run_agg(False))
    with pytest.raises(AssertionError):
        _check_agg(_run_agg(True))
