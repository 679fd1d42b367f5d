"""Graph parity (Sec. 2 of arXiv:1904.06257): the CUDA multispin graph kernel
against the CPU oracle.  Integer couplings: bit-exact trajectories (the fp32
fast path with its fp64 fallback must agree with the exact threshold test).
Real couplings: every decision of the product kernel equals the oracle's fp64
decision outside the band a field error of 1e-6 (sum |J| + q + |lambda|) can move,
and stationary observables agree within 4 standard errors."""
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
                             1.0, beta, seed, 0, 5, draw=core.DRAW_PLANE)
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
                          0.5, seed, 0, 0, beta_sched=sched, draw=core.DRAW_PLANE)
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


def _field_band(h, beta, scale):
    """Half-width (in units of the 32-bit draw) of the band around the heat-bath
    boundary 2^32 p(h), p = 1 / (1 + e^{-2 beta h}), inside which a correct fp32
    decision may differ from the fp64 one: a field error of 1e-6 * scale (the
    tolerance on real couplings, scale = sum |J| + q + |lambda|), the kernel's
    ex2.approx (relative 2^-22) and the rounding of its exponent (relative 2^-24 of
    2 beta h log2 e), the draw converted to fp32 and the product (2 x 2^-24 of 2^32 p),
    plus one unit for the floor."""
    with np.errstate(over="ignore"):  # p -> 0 for strongly negative fields
        p = 1.0 / (1.0 + np.exp(-2.0 * beta * h))
    dp = p * (1.0 - p)
    return (2.0 ** 32 * dp * (2.0 * beta * 1e-6 * scale + 2.0 ** -22
                              + np.abs(2.0 * beta * h) * 2.0 ** -23)
            + 2.0 ** 9 * p + 2.0), 2.0 ** 32 * p


def _half_types(reversed_):
    return (1, 0) if reversed_ else (0, 1)


@pytest.mark.parametrize("reversed_", [False, True])
def test_real_coupling_decisions_outside_field_band(S, reversed_):
    """The real-coupling product kernel (fp32 field sums and fp32 decision) against the
    oracle's fp64 fields and thresholds, every (vertex, replica) of both half steps of
    one full step: tau must equal the oracle's decision wherever the draw lies outside
    the band a field error of 1e-6 (sum |J| + q + |lambda|) can move (Sec. 2, the
    fields below Eq. (ham21) and the heat-bath half-step laws), and few lanes may lie
    inside it.  Each half step is checked from the GPU's own input configuration."""
    n, R, q = 10_000, 256, 1.0
    u, v, J, lam = er_instance(n, 8.0, 44, integer=False)
    beta = W.beta_grid(R, 0.2, 2.5, 64)
    seed = 8 + int(reversed_)
    ctx = S.shaken_init(graph_problem(S, n, u, v, J, R, beta, q=q, lam=lam, integer=False), seed)
    S.shaken_set_order(ctx, reversed_)
    S.shaken_step(ctx, 2)
    sig0 = S.shaken_get_spins(ctx, R, n)
    S.shaken_step(ctx, 1)
    sigp = S.shaken_get_spins_prime(ctx, R, n)
    sig1 = S.shaken_get_spins(ctx, R, n)
    S.shaken_free(ctx)
    tail, head = core.orient(u, v, 0)
    Jd, ld = J.astype(np.float64), lam.astype(np.float64)
    absJ = np.abs(Jd)
    t = 2
    total_in_band = 0
    for typ, src, out in zip(_half_types(reversed_), (sig0, sigp), (sigp, sig1)):
        h = core.graph_fields(src, tail, head, Jd, False, ld, q, typ)
        ref = core.graph_half(src, tail, head, Jd, False, ld, q, beta, seed, t, typ)
        draws = core.graph_draws(seed, n, R, t, typ, core.DRAW_DIRECT).astype(np.float64)
        ends = head if typ == 0 else tail  # the vertex whose field an edge enters
        scale = (np.bincount(ends, weights=absJ, minlength=n) + q + np.abs(ld))[None, :]
        band, bound = _field_band(h, beta[:, None], scale)
        outside = np.abs(draws - bound) > band
        bad = outside & (out != ref)
        assert not bad.any(), (typ, np.argwhere(bad)[:5])
        total_in_band += int((~outside).sum())
    # the band is a few parts in 10^6 of the draw range: a handful of lanes at most
    assert total_in_band <= 2e-4 * 2 * n * R, total_in_band


def _real_band_check(S, n, u, v, J, lam, R, beta, q, seed, orientation):
    """One full step of the real-coupling product kernel from a given orientation;
    returns the number of (vertex, replica) lanes inside the field band after
    asserting every lane outside it equals the oracle's fp64 decision."""
    ctx = S.shaken_init(graph_problem(S, n, u, v, J, R, beta, q=q, lam=lam, integer=False,
                                      orientation=orientation), seed)
    S.shaken_step(ctx, 1)
    sig0 = S.shaken_get_spins(ctx, R, n)
    S.shaken_step(ctx, 1)
    sigp = S.shaken_get_spins_prime(ctx, R, n)
    sig1 = S.shaken_get_spins(ctx, R, n)
    S.shaken_free(ctx)
    tail, head = core.orient(u, v, orientation)
    Jd, ld = J.astype(np.float64), lam.astype(np.float64)
    in_band = 0
    for typ, src, out in ((0, sig0, sigp), (1, sigp, sig1)):
        h = core.graph_fields(src, tail, head, Jd, False, ld, q, typ)
        ref = core.graph_half(src, tail, head, Jd, False, ld, q, beta, seed, 1, typ)
        draws = core.graph_draws(seed, n, R, 1, typ, core.DRAW_DIRECT).astype(np.float64)
        ends = head if typ == 0 else tail
        scale = (np.bincount(ends, weights=np.abs(Jd), minlength=n) + q + np.abs(ld))[None, :]
        band, bound = _field_band(h, beta[:, None], scale)
        outside = np.abs(draws - bound) > band
        bad = outside & (out != ref)
        assert not bad.any(), (orientation, typ, np.argwhere(bad)[:5])
        in_band += int((~outside).sum())
    return in_band


def test_real_coupling_hub_decisions_outside_field_band(S):
    """Vertices of degree above 255 with real couplings (the chunked hub kernel: per
    chunk fp32 sums, added in chunk order): a star with 10^4 leaves (its centre's
    edges in five chunks) with the centre on the in- and then the out-side, and a
    power-law graph (n = 20000, exponent 2.5, a dozen hubs) in both orientations.
    Every (vertex, replica) decision of both half steps equals the oracle's fp64
    decision outside the field band (Sec. 2, fields below Eq. (ham21))."""
    R, q = 64, 1.0
    leaves = 10_000
    n = leaves + 1
    src = np.arange(1, n, dtype=np.int32)
    hub = np.zeros(leaves, np.int32)
    J = W.couplings_normal(leaves, 21)
    lam = W.fields_normal(n, 0.1, 22)
    beta = W.beta_grid(R, 0.001, 0.02, 23)  # the centre's field is ~N(0, 10^4)
    in_band = 0
    for k, (uu, vv) in enumerate(((src, hub), (hub, src))):
        in_band += _real_band_check(S, n, uu, vv, J, lam, R, beta, q, 31 + k, 2)
    n = 20000
    u, v = W.power_law(n, 6.0, 2.5, 3)
    J = W.couplings_normal(u.size, 24)
    lam = W.fields_normal(n, 0.1, 25)
    beta = W.beta_grid(R, 0.05, 1.0, 26)
    for k, (uu, vv) in enumerate(((u, v), (v, u))):
        in_band += _real_band_check(S, n, uu, vv, J, lam, R, beta, q, 41 + k, 2)
    assert in_band <= 2e-4 * 2 * R * (leaves + 1 + n) * 2, in_band


def test_real_coupling_decisions_full_size_sampled(S):
    """The same check on the graph workload's size (Erdos-Renyi n = 10^6, mean degree
    8, J ~ N(0, 1) fp32, lambda_x ~ N(0, 0.1^2), q = 1, 256 replicas), at sampled
    (vertex, replica) pairs of both half steps, fields evaluated one vertex at a time
    by the oracle."""
    n, R, q = 1_000_000, 256, 1.0
    u, v = W.erdos_renyi(n, 8.0, W.BASE_SEED + 1)
    J = W.couplings_normal(u.size, W.BASE_SEED + 2)
    lam = W.fields_normal(n, 0.1, W.BASE_SEED + 3)
    beta = W.beta_grid(R, 0.1, 3.0, 64)
    seed = W.BASE_SEED + 12
    ctx = S.shaken_init(graph_problem(S, n, u, v, J, R, beta, q=q, lam=lam, integer=False), seed)
    S.shaken_step(ctx, 1)
    sig0 = S.shaken_get_spins(ctx, R, n)
    S.shaken_step(ctx, 1)
    sigp = S.shaken_get_spins_prime(ctx, R, n)
    sig1 = S.shaken_get_spins(ctx, R, n)
    S.shaken_free(ctx)
    tail, head = core.orient(u, v, 0)
    Jd, ld = J.astype(np.float64), lam.astype(np.float64)
    t = 1
    g = np.random.default_rng(33)
    in_band = 0
    for typ, src, out in ((0, sig0, sigp), (1, sigp, sig1)):
        inc = core.Incidence(n, tail, head, Jd, False, ld, q, typ)
        ends = head if typ == 0 else tail
        scale_all = np.bincount(ends, weights=np.abs(Jd), minlength=n) + q + np.abs(ld)
        for _ in range(400):
            x, r = int(g.integers(n)), int(g.integers(R))
            h = inc.field(src[r], x)
            tau = inc.site(src[r], x, r, beta[r], seed, t, core.DRAW_DIRECT)
            uu = core.graph_draw(seed, x, r, t, typ, core.DRAW_DIRECT)
            band, bound = _field_band(np.array(h), beta[r], scale_all[x])
            if abs(uu - bound) > band:
                assert out[r, x] == tau, (typ, x, r)
            else:
                in_band += 1
    assert in_band <= 2


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


def _hub_instance(n, seed):
    # Erdos-Renyi plus an in-hub: vertex n - 1 joined to every other vertex (under
    # min -> max orientation its n - 1 edges all enter it: two chunks of the hub kernel)
    u, v = W.erdos_renyi(n, 4.0, seed)
    a = np.concatenate([u, np.arange(n - 1)]).astype(np.int64)
    b = np.concatenate([v, np.full(n - 1, n - 1)]).astype(np.int64)
    keys = np.unique(np.minimum(a, b) * n + np.maximum(a, b))
    u, v = (keys // n).astype(np.int32), (keys % n).astype(np.int32)
    return u, v, W.couplings_pm1(u.size, seed + 1), W.fields_normal(n, 0.1, seed + 2)


@pytest.mark.parametrize("kind", ["er", "hub"])
def test_fused_tracking_best_energy(S, kind):
    # the best energy tracked inside half 0 (the hub kernel adds the words of vertices
    # of degree above 255) equals the minimum over steps of the oracle's H(sigma_t)
    # along the same (bit-exact) trajectory
    n, R = (500, 32) if kind == "er" else (3001, 64)
    u, v, J, lam = er_instance(n, 6.0, 91) if kind == "er" else _hub_instance(n, 95)
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
        cur, _ = core.graph_run(cur, tail, head, Jd, True, ld, 1.0, b, seed, k, 1,
                                draw=core.DRAW_PLANE)
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
        uu = core.graph_draw(seed, x, r, t, half, core.DRAW_PLANE)
        return 1 if uu < T else -1

    g = np.random.default_rng(21)
    for _ in range(150):
        x, r = int(g.integers(n)), int(g.integers(R))
        sr = s0[r].copy()
        ys = head[order_out[out_ptr[x]:out_ptr[x + 1]]]
        for y in list(ys) + [x]:  # sigma' where the second half step reads it
            sr[y] = site(s0[r], int(y), 0, r)
        assert s1[r, x] == site(sr, x, 1, r), (x, r)


@pytest.mark.parametrize("n,deg,R,q,beta", [(2000, 12.0, 64, 0.8, 0.7),   # classes (a, sigma)
                                             (1500, 30.0, 32, 1.0, 0.3),   # collapsed, d <= 30
                                             (1200, 5.0, 96, 1.0, 1.1)])   # collapsed, 3 groups
def test_integer_graph_class_tables_bit_exact(S, n, deg, R, q, beta):
    """One beta on every replica: the per-vertex class tables decide the lanes (class
    (a, sigma) tables for q != 1; with q = 1 the collapsed tables over a + sigma, since
    h(a, +1) = h(a + 1, -1) exactly), at every table width (degrees up to 7, 15, 31)
    and above them through per-lane thresholds; bit-exact against the oracle."""
    u, v, J, lam = er_instance(n, deg, 300 + n, lam_sd=0.2)
    seed = 0x5348414B + 7 * n
    ctx = S.shaken_init(graph_problem(S, n, u, v, J, R, beta, q=q, lam=lam), seed)
    S.shaken_step(ctx, 3)
    got = S.shaken_get_spins(ctx, R, n)
    S.shaken_free(ctx)
    tail, head = core.orient(u, v, 0)
    o = core.graph_init(n, R, seed, 0)
    o, _ = core.graph_run(o, tail, head, J.astype(np.float64), True, lam.astype(np.float64), q,
                          beta, seed, 0, 3, draw=core.DRAW_PLANE)
    assert np.array_equal(got, o)


@pytest.mark.parametrize("integer", [True, False])
def test_graph_step_record_series(S, integer):
    """The per-step series of a graph context (shaken_step_record: m and H(sigma_t) of
    every replica at every step, from the graph observables kernel) against the
    oracle's observables of the oracle's trajectory: m exactly, H within 1e-6 of its
    scale sum |J| + 2 sum |lambda| (the scale of the fp32 sums, as for the fields).  Real
    couplings: only the first step is compared (the trajectories agree outside the
    field band, not bit for bit)."""
    n, R, steps = 600, 64, 6 if integer else 1
    u, v, J, lam = er_instance(n, 6.0, 91, integer=integer)
    beta = W.beta_grid(R, 0.3, 1.5, 64)
    seed = 93
    ctx = S.shaken_init(graph_problem(S, n, u, v, J, R, beta, q=1.0, lam=lam,
                                      integer=integer), seed)
    mag, en = S.shaken_step_record(ctx, steps, R)
    S.shaken_free(ctx)
    tail, head = core.orient(u, v, 0)
    Jd, ld = J.astype(np.float64), lam.astype(np.float64)
    cur = core.graph_init(n, R, seed, 0)
    scale = np.abs(Jd).sum() + 2.0 * np.abs(ld).sum()
    for k in range(steps):
        ref = core.graph_observables(cur, cur, tail, head, Jd, ld, 1.0)
        for r in range(R):
            assert abs(mag[k, r] - ref[r]["m"]) < 1e-12, (k, r)
            assert abs(en[k, r] - ref[r]["H"]) < 1e-6 * (abs(ref[r]["H"]) + scale), (k, r)
        cur, _ = core.graph_run(cur, tail, head, Jd, integer, ld, 1.0, beta, seed, k, 1,
                                draw=core.DRAW_PLANE if integer else core.DRAW_DIRECT)


@pytest.mark.parametrize("reverse", [False, True])
def test_graph_observables_with_hubs(S, reverse):
    """Observables of a graph with a vertex of degree 3000 (the observables kernel
    counts its edges in chunks of 252 per thread) against the oracle's, in both
    orientations of the hub's edges: m and cut exactly, H and the pair energy within
    1e-6 rel (integer couplings, fp32 lambda sums)."""
    n, R = 3001, 64
    u, v, J, lam = _hub_instance(n, 97)
    orientation = 0
    if reverse:  # the hub's edges leave it: given orientation, hub as the tail
        u, v = np.where(v == n - 1, v, u), np.where(v == n - 1, u, v)
        orientation = 2
    beta = W.beta_grid(R, 0.2, 1.5, 64)
    seed = 99
    ctx = S.shaken_init(graph_problem(S, n, u, v, J, R, beta, q=1.0, lam=lam,
                                      orientation=orientation), seed)
    S.shaken_step(ctx, 3)
    s1 = S.shaken_get_spins(ctx, R, n)
    sp = S.shaken_get_spins_prime(ctx, R, n)
    obs = S.shaken_observables(ctx, R)
    S.shaken_free(ctx)
    tail, head = core.orient(u, v, orientation)
    ref = core.graph_observables(s1, sp, tail, head, J.astype(np.float64),
                                 lam.astype(np.float64), 1.0)
    for r in range(R):
        assert abs(obs["magnetization"][r] - ref[r]["m"]) < 1e-12
        assert abs(obs["energy"][r] - ref[r]["H"]) < 1e-6 * (1 + abs(ref[r]["H"]))
        assert abs(obs["pair_energy"][r] - ref[r]["pair"]) < 1e-6 * (1 + abs(ref[r]["pair"]))
        assert obs["cut_edges"][r] == ref[r]["cut"]
