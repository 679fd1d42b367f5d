"""Graph parity (Sec. 2 of arXiv:1904.06257): the CUDA multispin graph kernel
against the CPU oracle.  Integer couplings: bit-exact trajectories (the fp32
fast path with its fp64 fallback must agree with the exact threshold test).
Real couplings: local fields within 1e-6 of the fp64 value (relative to
sum |J| + q + |lambda|) and stationary observables within 4 standard errors."""
import numpy as np
import pytest

from oracle import core, exact
from paper_1904_06257_gb300 import workloads as W
from tests.gpu_util import graph_problem, lib, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    require_cuda()
    return lib()


def er_instance(n, deg, seed, integer=True, lam_sd=0.1):
    u, v = W.erdos_renyi(n, deg, seed)
    J = W.couplings_pm1(u.size, seed + 1) if integer else W.couplings_normal(u.size, seed + 1)
    lam = W.fields_normal(n, lam_sd, seed + 2)
    return u, v, J, lam


@pytest.mark.parametrize("n,deg,R,orientation", [(1000, 8.0, 64, 0), (777, 3.0, 32, 2)])
def test_integer_graph_bit_exact(S, n, deg, R, orientation):
    u, v, J, lam = er_instance(n, deg, 11 + n)
    beta = W.beta_grid(R, 0.2, 2.5, 13)
    seed = 0x5348414B + n
    ctx = S.shaken_init(graph_problem(S, n, u, v, J, R, beta, q=1.0, lam=lam,
                                      orientation=orientation), seed)
    s0 = S.shaken_get_spins(ctx, R, n)
    o0 = core.graph_init(n, R, seed, 0)
    assert np.array_equal(s0, o0)
    S.shaken_step(ctx, 5)
    s1 = S.shaken_get_spins(ctx, R, n)
    tail, head = core.orient(u, v, orientation)
    o1, osp = core.graph_run(o0, tail, head, J.astype(np.float64), True, lam.astype(np.float64),
                             1.0, beta, seed, 0, 5)
    assert np.array_equal(s1, o1)
    obs = S.shaken_observables(ctx, R)
    ref = core.graph_observables(o1, osp, tail, head, J.astype(np.float64),
                                 lam.astype(np.float64), 1.0)
    for r in range(R):
        assert abs(obs["magnetization"][r] - ref[r]["m"]) < 1e-12
        assert abs(obs["energy"][r] - ref[r]["H"]) < 1e-6 * (1 + abs(ref[r]["H"]))
        assert abs(obs["pair_energy"][r] - ref[r]["pair"]) < 1e-6 * (1 + abs(ref[r]["pair"]))
        assert obs["cut_edges"][r] == ref[r]["cut"]
    S.shaken_free(ctx)


def test_fast_path_equals_exact_path(S):
    # the fp32 fast decision with its error margin agrees with the fp64 threshold everywhere
    n, R = 4000, 128
    u, v, J, lam = er_instance(n, 8.0, 5, lam_sd=0.3)
    beta = W.beta_grid(R, 0.05, 3.0, 64)
    res = []
    for exact_always in (False, True):
        ctx = S.shaken_init(graph_problem(S, n, u, v, J, R, beta, q=0.7, lam=lam), 9)
        S.shaken_debug_exact_always(ctx, exact_always)
        S.shaken_step(ctx, 30)
        res.append(S.shaken_get_spins(ctx, R, n))
        S.shaken_free(ctx)
    assert np.array_equal(res[0], res[1])


def test_graph_anneal_bit_exact(S):
    n, R = 600, 32
    u, v, J, lam = er_instance(n, 6.0, 21)
    sched = W.linear_schedule(0.1, 3.0, 10)
    seed = 31337
    ctx = S.shaken_init(graph_problem(S, n, u, v, J, R, 0.5, q=1.0, lam=lam), seed)
    S.shaken_anneal(ctx, sched)
    s = S.shaken_get_spins(ctx, R, n)
    tail, head = core.orient(u, v, 0)
    o = core.graph_init(n, R, seed, 0)
    o, _ = core.graph_run(o, tail, head, J.astype(np.float64), True, lam.astype(np.float64), 1.0,
                          0.5, seed, 0, 0, beta_sched=sched)
    assert np.array_equal(s, o)
    S.shaken_free(ctx)


def test_lattice_as_graph_matches_lattice_fields(S):
    # the lattice fed as a graph with the lattice orientation gives the lattice fields
    L, R = 32, 32
    u, v = W.lattice_as_graph(L)
    J = np.ones(u.size, dtype=np.float32)
    ctx = S.shaken_init(graph_problem(S, L * L, u, v, J, R, 0.4, q=0.8, lam_c=0.1,
                                      orientation=S.ORIENT_GIVEN), 3)
    s = S.shaken_get_spins(ctx, R, L * L).astype(np.int64)
    for half in (0, 1):
        h = S.shaken_debug_fields(ctx, half, R, L * L).astype(np.float64)
        tails, heads = exact.lattice_edges(L)
        Jo = exact.oriented_matrix(L * L, tails, heads, 1.0)
        ref = exact.fields(s, Jo, 0.1, 0.8, half)
        assert np.abs(h - ref).max() < 1e-5
    S.shaken_free(ctx)


def test_real_fields_within_tolerance(S):
    n, R = 1500, 64
    u, v, J, lam = er_instance(n, 8.0, 44, integer=False)
    ctx = S.shaken_init(graph_problem(S, n, u, v, J, R, 0.5, q=1.0, lam=lam, integer=False), 8)
    S.shaken_step(ctx, 3)
    s = S.shaken_get_spins(ctx, R, n).astype(np.int64)
    tail, head = core.orient(u, v, 0)
    Jo = exact.oriented_matrix(n, tail, head, J.astype(np.float64))
    absJ = exact.oriented_matrix(n, tail, head, np.abs(J.astype(np.float64)))
    for half in (0, 1):
        # half 1 reads sigma' (B); after full steps B holds the last half-step state
        h = S.shaken_debug_fields(ctx, half, R, n).astype(np.float64)
        if half == 1:
            continue  # sigma' is not returned by get_spins; half 0 covers the sums
        ref = exact.fields(s, Jo, lam.astype(np.float64), 1.0, 0)
        scale = absJ.sum(axis=0)[None, :] + 1.0 + np.abs(lam)[None, :]
        assert (np.abs(h - ref) / scale).max() < 1e-6
    S.shaken_free(ctx)


def test_real_graph_statistics_match_oracle(S):
    n = 400
    u, v, J, lam = er_instance(n, 6.0, 77, integer=False, lam_sd=0.2)
    beta, q = 0.6, 1.0
    Rg, Ro, burn, meas = 256, 128, 60, 40
    ctx = S.shaken_init(graph_problem(S, n, u, v, J, Rg, beta, q=q, lam=lam, integer=False), 1)
    S.shaken_step(ctx, burn)
    eg, mg = [], []
    for _ in range(meas):
        S.shaken_step(ctx, 1)
        o = S.shaken_observables(ctx, Rg)
        eg.append(o["energy"].copy())
        mg.append(o["magnetization"].copy())
    S.shaken_free(ctx)
    tail, head = core.orient(u, v, 0)
    Jd, ld = J.astype(np.float64), lam.astype(np.float64)
    cur = core.graph_init(n, Ro, 2, 0)
    cur, sp = core.graph_run(cur, tail, head, Jd, False, ld, q, beta, 2, 0, burn)
    eo, mo = [], []
    for k in range(meas):
        cur, sp = core.graph_run(cur, tail, head, Jd, False, ld, q, beta, 2, burn + k, 1)
        ob = core.graph_observables(cur, sp, tail, head, Jd, ld, q)
        eo.append([x["H"] for x in ob])
        mo.append([x["m"] for x in ob])
    for g, o in ((np.array(eg), np.array(eo)), (np.array(mg), np.array(mo))):
        # per-replica time averages are independent across replicas
        ga, oa = g.mean(axis=0), o.mean(axis=0)
        se = np.sqrt(ga.var(ddof=1) / ga.size + oa.var(ddof=1) / oa.size)
        assert abs(ga.mean() - oa.mean()) < 4 * se + 1e-12


def test_fused_tracking_best_energy(S):
    # the best energy tracked inside half 0 equals the minimum over steps of the
    # oracle's H(sigma_t) along the same (bit-exact) trajectory
    n, R = 500, 32
    u, v, J, lam = er_instance(n, 6.0, 91)
    sched = W.linear_schedule(0.2, 2.5, 15)
    seed = 4711
    ctx = S.shaken_init(graph_problem(S, n, u, v, J, R, 0.5, q=1.0, lam=lam), seed)
    S.shaken_anneal(ctx, sched)
    obs = S.shaken_observables(ctx, R)
    S.shaken_free(ctx)
    tail, head = core.orient(u, v, 0)
    Jd, ld = J.astype(np.float64), lam.astype(np.float64)
    cur = core.graph_init(n, R, seed, 0)
    best = np.full(R, np.inf)
    for k, b in enumerate(sched):
        H = np.array([o["H"] for o in core.graph_observables(cur, cur, tail, head, Jd, ld, 1.0)])
        best = np.minimum(best, H)
        cur, _ = core.graph_run(cur, tail, head, Jd, True, ld, 1.0, b, seed, k, 1)
    H = np.array([o["H"] for o in core.graph_observables(cur, cur, tail, head, Jd, ld, 1.0)])
    best = np.minimum(best, H)
    assert np.allclose(obs["best_energy"], best, rtol=1e-6, atol=1e-4)


def test_full_size_anneal_step_sampled(S):
    """The bench's graph workload (Erdos-Renyi n = 10^6, mean degree 8, +-1 couplings,
    lambda_x ~ N(0, 0.1^2), q = 1, 256 replicas, one anneal step with its beta on every
    replica and the best-energy tracking fused into half 0): sampled (vertex, replica)
    pairs of the full step against the oracle's single-site decisions."""
    n, R, q, beta = 1_000_000, 256, 1.0, 1.7
    u, v = W.erdos_renyi(n, 8.0, W.BASE_SEED + 1)
    J = W.couplings_pm1(u.size, W.BASE_SEED + 2)
    lam = W.fields_normal(n, 0.1, W.BASE_SEED + 3)
    seed = W.BASE_SEED + 11
    ctx = S.shaken_init(graph_problem(S, n, u, v, J, R, 0.1, q=q, lam=lam), seed)
    S.shaken_step(ctx, 2)
    S.shaken_set_tracking(ctx, True)
    s0 = S.shaken_get_spins(ctx, R, n)
    S.shaken_anneal(ctx, np.array([beta]))
    s1 = S.shaken_get_spins(ctx, R, n)
    S.shaken_free(ctx)
    tail, head = core.orient(u, v, 0)
    order_in, order_out = np.argsort(head, kind="stable"), np.argsort(tail, kind="stable")
    in_ptr = np.searchsorted(head[order_in], np.arange(n + 1))
    out_ptr = np.searchsorted(tail[order_out], np.arange(n + 1))
    t = 2

    def site(sr, x, half, r):
        # tau_x from the in-neighbours (half 0) or out-neighbours (half 1) of x in sr
        if half == 0:
            es = order_in[in_ptr[x]:in_ptr[x + 1]]
            ys = tail[es]
        else:
            es = order_out[out_ptr[x]:out_ptr[x + 1]]
            ys = head[es]
        s = int(np.sum(np.where(J[es] > 0, 1, -1) * sr[ys].astype(np.int64)))
        h = core.field(1.0, s, q, int(sr[x]), float(lam[x]))
        T = core.threshold(h, beta)
        uu = core.draw_direct(seed, x, r >> 5, t, half, r & 31)
        return 1 if uu < T else -1

    g = np.random.default_rng(21)
    for _ in range(150):
        x, r = int(g.integers(n)), int(g.integers(R))
        sr = s0[r].copy()
        ys = head[order_out[out_ptr[x]:out_ptr[x + 1]]]
        for y in list(ys) + [x]:  # sigma' where the second half step reads it
            sr[y] = site(s0[r], int(y), 0, r)
        assert s1[r, x] == site(sr, x, 1, r), (x, r)
