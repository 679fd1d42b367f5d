"""Runtime behaviour through the C ABI on the GPU: batching (uneven sizes in
one launch per half step, CUDA-graph replay) gives each member the trajectory
it has alone; checkpoint/resume is bit-exact; the serving loop's results equal
running each job alone; the device Philox and thresholds equal the oracle's."""
import numpy as np
import pytest

from oracle import core
from paper_1904_06257_gb300 import workloads as W
from tests.gpu_util import graph_problem, graph_spins_from_raw, lattice_problem, lib, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    require_cuda()
    return lib()


def make_members(S):
    u, v = W.erdos_renyi(700, 5.0, 3)
    J = W.couplings_pm1(u.size, 4)
    lam = W.fields_normal(700, 0.1, 5)
    probs = [
        (lattice_problem(S, S.INT8, 64, 2, [0.4, 0.5]), 1, 64 * 64, 2),
        (lattice_problem(S, S.PACKED, 96, 1, 0.44, lam=0.01), 2, 96 * 96, 1),
        (lattice_problem(S, S.MULTISPIN, 32, 32, W.beta_grid(32)), 3, 32 * 32, 32),
        (lattice_problem(S, S.MULTISPIN, 128, 64, W.beta_grid(64)), 4, 128 * 128, 64),
        (graph_problem(S, 700, u, v, J, 32, 0.8, lam=lam), 5, 700, 32),
    ]
    return probs


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_alone(S, use_graph):
    steps = 70
    alone = []
    for p, seed, n, R in make_members(S):
        c = S.shaken_init(p, seed)
        S.shaken_step(c, steps)
        alone.append(S.shaken_get_spins(c, R, n))
        S.shaken_free(c)
    b = S.shaken_batch_create()
    ctxs = []
    for p, seed, n, R in make_members(S):
        c = S.shaken_init(p, seed)
        S.shaken_batch_add(b, c)
        ctxs.append((c, n, R))
    S.shaken_batch_step(b, steps, use_graph)
    S.shaken_batch_sync(b)
    assert S.shaken_batch_launch_count(b) > 0
    for (c, n, R), ref in zip(ctxs, alone):
        assert np.array_equal(S.shaken_get_spins(c, R, n), ref)
        assert S.shaken_get_step(c) == steps
    for c, _, _ in ctxs:
        S.shaken_batch_remove(b, c)
        S.shaken_free(c)
    S.shaken_batch_free(b)


def test_batch_of_hub_graphs_equals_alone_and_oracle(S):
    """Graph contexts whose vertices of degree above 255 go to the chunked hub kernel,
    batched together (one family: the hub chunks of several jobs, different group
    counts, one context in reversed step order so its half steps take the other
    direction's hubs first): every member equals its run alone and the oracle."""
    n1 = 3001  # star: centre 0 with 3000 leaves (two chunks of 2048 edges)
    u1 = np.zeros(n1 - 1, np.int32)
    v1 = np.arange(1, n1, dtype=np.int32)
    J1 = W.couplings_pm1(n1 - 1, 51)
    lam1 = W.fields_normal(n1, 0.2, 52)
    n2 = 20000
    u2, v2 = W.power_law(n2, 6.0, 2.5, 53)
    J2 = W.couplings_pm1(u2.size, 54)
    lam2 = W.fields_normal(n2, 0.1, 55)
    members = [  # (problem args, seed, R, reversed)
        ((n1, u1, v1, J1, 64, W.beta_grid(64, 0.01, 0.05, 64), 0.5, lam1), 61, 64, False),
        ((n2, u2, v2, J2, 32, 0.7, 1.0, lam2), 62, 32, False),
        ((n2, u2, v2, J2, 96, W.beta_grid(96, 0.3, 1.2, 57), 1.0, lam2), 63, 96, True),
    ]
    steps = 6

    def make(args, seed, rev):
        n, u, v, J, R, beta, q, lam = args
        c = S.shaken_init(graph_problem(S, n, u, v, J, R, beta, q=q, lam=lam), seed)
        if rev:
            S.shaken_set_order(c, True)
        return c

    alone = []
    for args, seed, R, rev in members:
        c = make(args, seed, rev)
        S.shaken_step(c, steps)
        alone.append(S.shaken_get_spins(c, R, args[0]))
        S.shaken_free(c)
    b = S.shaken_batch_create()
    ctxs = []
    for args, seed, R, rev in members:
        c = make(args, seed, rev)
        S.shaken_batch_add(b, c)
        ctxs.append(c)
    S.shaken_batch_step(b, steps, False)
    S.shaken_batch_sync(b)
    for c, ref, (args, seed, R, rev) in zip(ctxs, alone, members):
        got = S.shaken_get_spins(c, R, args[0])
        assert np.array_equal(got, ref), seed
        n, u, v, J, R_, beta, q, lam = args
        tail, head = core.orient(u, v, 0)
        o = core.graph_init(n, R, seed, 0)
        for t in range(steps):
            for typ in ((1, 0) if rev else (0, 1)):
                o = core.graph_half(o, tail, head, J.astype(np.float64), True,
                                    lam.astype(np.float64), q, beta, seed, t, typ,
                                    draw=core.DRAW_PLANE)
        assert np.array_equal(got, o), seed
    for c in ctxs:
        S.shaken_batch_remove(b, c)
        S.shaken_free(c)
    S.shaken_batch_free(b)


def test_batch_observables_and_async_state_equal_per_context_calls(S):
    """shaken_batch_observables (one launch per family for all members) gives each
    member's records exactly as shaken_observables on the same states, in member
    order; shaken_get_state_raw_async gives the bytes of shaken_get_state_raw; the
    packed batch copies (one transfer for all members) agree with both."""
    import torch
    b = S.shaken_batch_create()
    ctxs = []
    for p, seed, n, R in make_members(S):
        c = S.shaken_init(p, seed)
        S.shaken_batch_add(b, c)
        ctxs.append((c, R))
    S.shaken_batch_step(b, 9, False)
    total = sum(R for _, R in ctxs)
    sizes = [S.shaken_state_bytes(c) for c, _ in ctxs]
    bufs = [torch.zeros(n, dtype=torch.uint8, pin_memory=True) for n in sizes]
    for (c, _), buf, n in zip(ctxs, bufs, sizes):
        S.shaken_get_state_raw_async(c, buf.data_ptr(), n)
    batched = S.shaken_batch_observables(b, total)
    off = 0
    for (c, R), buf, n in zip(ctxs, bufs, sizes):
        ref = torch.zeros(n, dtype=torch.uint8, pin_memory=True)
        S.shaken_get_state_raw(c, ref.data_ptr(), n)
        assert torch.equal(buf, ref)
        single = S.shaken_observables(c, R)
        for f in ("magnetization", "energy", "pair_energy", "cut_edges", "cut_weight"):
            assert np.array_equal(batched[f][off:off + R], single[f]), f
        off += R
    assert off == total
    # all states in one transfer each way: equal to the per-context raw copies, and
    # a second batch loaded from them holds the same states
    tot = S.shaken_batch_state_bytes(b)
    assert tot == sum(sizes)
    packed = torch.zeros(tot, dtype=torch.uint8, pin_memory=True)
    S.shaken_batch_get_states_raw_async(b, packed.data_ptr(), tot)
    S.shaken_batch_sync(b)
    assert torch.equal(packed, torch.cat(bufs))
    b2 = S.shaken_batch_create()
    ctxs2 = []
    for p, seed, n, R in make_members(S):
        c = S.shaken_init(p, seed + 100)
        S.shaken_batch_add(b2, c)
        ctxs2.append(c)
    S.shaken_batch_set_states_raw(b2, packed.data_ptr(), tot)
    S.shaken_batch_sync(b2)
    for c, buf, n in zip(ctxs2, bufs, sizes):
        got = torch.zeros(n, dtype=torch.uint8, pin_memory=True)
        S.shaken_get_state_raw(c, got.data_ptr(), n)
        assert torch.equal(got, buf)
    # size mismatches and a negative timing stride are rejected
    with pytest.raises(S.ShakenError):
        S.shaken_batch_set_states_raw(b2, packed.data_ptr(), tot - 4)
    with pytest.raises(S.ShakenError):
        S.shaken_batch_get_states_raw_async(b2, packed.data_ptr(), tot + 4)
    with pytest.raises(S.ShakenError):
        S.shaken_batch_set_timing(b2, -1)
    # timing every step vs a stride of 3 (steps 0 and 3 of 5): 2/5 of the launches
    S.shaken_batch_set_timing(b2, 1)
    S.shaken_batch_step(b2, 5, False)
    ms1, n1 = S.shaken_batch_kernel_time(b2)
    S.shaken_batch_set_timing(b2, 3)
    S.shaken_batch_step(b2, 5, False)
    ms3, n3 = S.shaken_batch_kernel_time(b2)
    S.shaken_batch_set_timing(b2, 0)
    assert n1 > 0 and n1 % 10 == 0 and n3 * 5 == n1 * 2 and ms1 > 0.0 and ms3 > 0.0
    for c in ctxs2:
        S.shaken_batch_remove(b2, c)
        S.shaken_free(c)
    S.shaken_batch_free(b2)
    for c, _ in ctxs:
        S.shaken_batch_remove(b, c)
        S.shaken_free(c)
    S.shaken_batch_free(b)


def test_checkpoint_resume_bit_exact(S):
    p = lattice_problem(S, S.MULTISPIN, 64, 32, W.beta_grid(32))
    c = S.shaken_init(p, 12)
    S.shaken_set_tracking(c, True)
    S.shaken_step(c, 10)
    ck = S.shaken_save(c)
    S.shaken_step(c, 15)
    ref = S.shaken_get_spins(c, 32, 64 * 64)
    ref_obs = S.shaken_observables(c, 32)
    c2 = S.shaken_init(p, 12)
    S.shaken_load(c2, ck)
    assert S.shaken_get_step(c2) == 10
    S.shaken_step(c2, 15)
    assert np.array_equal(S.shaken_get_spins(c2, 32, 64 * 64), ref)
    o2 = S.shaken_observables(c2, 32)
    assert np.array_equal(o2["best_energy"], ref_obs["best_energy"])
    S.shaken_free(c)
    S.shaken_free(c2)


def test_server_results_equal_alone(S):
    jobs = []
    for k in range(5):
        n = 300 + 150 * k
        u, v = W.erdos_renyi(n, 4.0 + k, 100 + k)
        J = W.couplings_pm1(u.size, 200 + k)
        lam = W.fields_normal(n, 0.1, 300 + k)
        R = 32 * (1 + k % 2)
        steps = 40 + 23 * k
        sched = W.linear_schedule(0.1, 3.0, steps)
        jobs.append((graph_problem(S, n, u, v, J, R, 1.0, lam=lam), 900 + k, sched, n, R))
    alone = []
    for p, seed, sched, n, R in jobs:
        c = S.shaken_init(p, seed)
        S.shaken_anneal(c, sched)
        alone.append((S.shaken_get_spins(c, R, n), S.shaken_observables(c, R)))
        S.shaken_free(c)
    srv = S.shaken_server_create(1 << 30, 16)
    S.shaken_server_set_policy(srv, 1.5e9, 0, keep_states=True)
    ids = [S.shaken_server_submit(srv, p, seed, sched) for p, seed, sched, n, R in jobs]
    S.shaken_server_drain(srv, 120.0)
    for jid, (p, seed, sched, n, R), (spins, obs) in zip(ids, jobs, alone):
        assert S.shaken_server_poll(srv, jid) == 2
        res, ta, td = S.shaken_server_result(srv, jid, R)
        assert td >= ta
        raw = S.shaken_server_result_state(srv, jid, R * n // 8)
        assert np.array_equal(graph_spins_from_raw(raw, n, R), spins)
        assert np.allclose(res["energy"], obs["energy"], rtol=0, atol=1e-9)
        # best energies are fp32 block sums added in a run-dependent order: equal to ~1e-6
        assert np.allclose(res["best_energy"], obs["best_energy"], rtol=1e-6, atol=1e-6)
    upd, launches, done = S.shaken_server_stats(srv)
    assert done == len(jobs) and launches > 0
    S.shaken_server_free(srv)


def test_server_work_cap_completes_jobs_under_overload(S):
    """Overload: twelve jobs at once, a work cap that admits about two at a time.  Jobs
    complete while others still wait (the queue is non-empty when the first results
    exist), every job completes, and each result equals the job run alone.  With
    shortest-work-first admission a small job submitted behind large ones finishes
    before them."""
    import time
    n = 3000
    u, v = W.erdos_renyi(n, 6.0, 71)
    J = W.couplings_pm1(u.size, 72)
    big = graph_problem(S, n, u, v, J, 64, 1.0)
    sched = W.linear_schedule(0.2, 2.5, 200)
    step_work = 2.0 * n * 64
    srv = S.shaken_server_create(1 << 30, 8)
    S.shaken_server_set_policy(srv, 2.5 * step_work, 0)
    ids = [S.shaken_server_submit(srv, big, 500 + k, sched) for k in range(12)]
    saw_queue_with_done = False
    t_end = time.perf_counter() + 120.0
    while time.perf_counter() < t_end:
        _, _, done = S.shaken_server_stats(srv)
        queued, running = S.shaken_server_queue(srv)
        assert running <= 2
        if done > 0 and queued > 0:
            saw_queue_with_done = True
        if done == len(ids):
            break
        time.sleep(0.002)
    S.shaken_server_drain(srv, 60.0)
    assert saw_queue_with_done
    c = S.shaken_init(big, 500)
    S.shaken_anneal(c, sched)
    ref = S.shaken_observables(c, 64)
    S.shaken_free(c)
    res, _, _ = S.shaken_server_result(srv, ids[0], 64)
    assert np.allclose(res["energy"], ref["energy"], rtol=0, atol=1e-9)
    S.shaken_server_free(srv)
    # shortest total work first: the small job overtakes the queued large ones
    small_n = 400
    su, sv = W.erdos_renyi(small_n, 4.0, 73)
    small = graph_problem(S, small_n, su, sv, W.couplings_pm1(su.size, 74), 32, 1.0)
    srv = S.shaken_server_create(1 << 30, 8)
    S.shaken_server_set_policy(srv, step_work, 1)  # one large job at a time
    large_ids = [S.shaken_server_submit(srv, big, 600 + k, sched) for k in range(4)]
    small_id = S.shaken_server_submit(srv, small, 700, W.linear_schedule(0.2, 2.5, 50))
    S.shaken_server_drain(srv, 120.0)
    t_small = S.shaken_server_result(srv, small_id, 32)[2]
    t_large = [S.shaken_server_result(srv, i, 64)[2] for i in large_ids]
    # done before every large job but the one that may already have been running
    assert t_small < sorted(t_large)[1]
    with pytest.raises(S.ShakenError):
        S.shaken_server_set_policy(srv, 0.0, 0)
    S.shaken_server_free(srv)


def test_server_budget_serialises_jobs(S):
    # a budget that fits one job at a time still completes every job
    n = 2000
    u, v = W.erdos_renyi(n, 6.0, 7)
    J = W.couplings_pm1(u.size, 8)
    p = graph_problem(S, n, u, v, J, 64, 1.0)
    srv = S.shaken_server_create(250_000, 8)  # one ~175 kB job fits at a time
    sched = W.linear_schedule(0.2, 2.0, 30)
    ids = [S.shaken_server_submit(srv, p, s, sched) for s in range(4)]
    S.shaken_server_drain(srv, 120.0)
    t = [S.shaken_server_result(srv, i, 64)[1:] for i in ids]
    for (a0, d0), (a1, d1) in zip(t, t[1:]):
        assert a1 >= d0 - 1e-9  # admitted only after the previous job freed its memory
    S.shaken_server_free(srv)


def test_device_philox_and_thresholds_match_oracle(S):
    import torch
    g = np.random.default_rng(0)
    n = 4096
    ctr = g.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    seed = 0x5348414B12345
    dc = torch.from_numpy(ctr.view(np.int32).copy()).cuda()
    do = torch.zeros_like(dc)
    S.shaken_philox_device(seed, dc.data_ptr(), do.data_ptr(), n)
    torch.cuda.synchronize()
    got = do.cpu().numpy().view(np.uint32)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    for i in range(0, n, 37):
        assert np.array_equal(got[i], core.philox(key, ctr[i]))
    h = np.concatenate([g.uniform(-10, 10, 20000), np.array([0.0, 7.0, -20.0, 1e-300]),
                        g.integers(-30, 30, 4000) + g.choice([-0.5, 0.0, 0.25, 0.5], 4000)])
    beta = np.concatenate([g.uniform(0, 3.5, h.size - 1), [100.0]])
    dh = torch.from_numpy(h).cuda()
    db = torch.from_numpy(beta).cuda()
    dout = torch.zeros(h.size, dtype=torch.int64, device="cuda")
    S.shaken_threshold_device(dh.data_ptr(), db.data_ptr(), dout.data_ptr(), h.size)
    torch.cuda.synchronize()
    T = dout.cpu().numpy().astype(np.uint64)
    for i in range(h.size):
        assert int(T[i]) == core.threshold(h[i], beta[i]), (h[i], beta[i])


def test_server_free_cancels_queued_and_running_jobs(S):
    # a job far too long to finish and one queued behind it (budget fits one job):
    # freeing the server stops after the current chunk and releases both
    import time
    n = 4000
    u, v = W.erdos_renyi(n, 6.0, 17)
    J = W.couplings_pm1(u.size, 18)
    p = graph_problem(S, n, u, v, J, 64, 1.0)
    srv = S.shaken_server_create(500_000, 8)  # one ~335 kB job fits at a time
    sched = W.linear_schedule(0.2, 2.0, 2_000_000)
    a = S.shaken_server_submit(srv, p, 1, sched)
    b = S.shaken_server_submit(srv, p, 2, sched)
    t_end = time.perf_counter() + 30.0
    while S.shaken_server_poll(srv, a) != 1 and time.perf_counter() < t_end:
        time.sleep(0.01)
    assert S.shaken_server_poll(srv, a) == 1   # running
    assert S.shaken_server_poll(srv, b) == 0   # queued behind it
    t0 = time.perf_counter()
    S.shaken_server_free(srv)
    assert time.perf_counter() - t0 < 10.0


def test_microbenchmarks(S):
    for kind in range(8):
        rate, ms = S.shaken_microbench(kind)
        assert rate > 0 and ms > 0
    for bad in (-1, 8):
        with pytest.raises(S.ShakenError):
            S.shaken_microbench(bad)
