"""Edge cases and degenerate inputs through the C ABI, against the oracle
(bit-exact unless stated): graphs without edges, isolated vertices, a vertex of
degree > 63 (the per-lane counting fallback), frozen vertices, beta = 0 (every
threshold 2^31), saturated thresholds, given orientations, the smallest and
large lattice sizes, and every initialisation kind."""
import numpy as np
import pytest

from oracle import core
from paper_1904_06257_gb300 import workloads as W
from tests.gpu_util import graph_problem, lattice_problem, lib, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    require_cuda()
    return lib()


def run_graph_both(S, n, u, v, J, R, beta, q, lam, steps, seed, integer=True, orientation=0,
                   frozen=None, init=0):
    ctx = S.shaken_init(graph_problem(S, n, u, v, J, R, beta, q=q, lam=lam, integer=integer,
                                      orientation=orientation, frozen=frozen, init=init), seed)
    S.shaken_step(ctx, steps)
    got = S.shaken_get_spins(ctx, R, n)
    S.shaken_free(ctx)
    tail, head = core.orient(u, v, orientation)
    o = core.graph_init(n, R, seed, init, frozen)
    o, _ = core.graph_run(o, tail, head, np.asarray(J, np.float64), integer,
                          np.asarray(lam, np.float64), q, beta, seed, 0, steps, frozen=frozen,
                          draw=core.DRAW_PLANE if integer else core.DRAW_DIRECT)
    return got, o


def test_graph_without_edges(S):
    n, R = 300, 32
    u = v = np.zeros(0, np.int32)
    J = np.zeros(0, np.float32)
    lam = W.fields_normal(n, 0.5, 1)
    got, ref = run_graph_both(S, n, u, v, J, R, 0.7, 0.9, lam, 4, 11)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("leaves", [100, 300])
def test_star_graph_high_degree_and_isolated(S, leaves):
    # vertex 0 joined to `leaves` leaves (in-degree 0 and out-degree `leaves` with
    # min->max; reversed orientation gives in-degree `leaves`: above 63, and 300 is
    # above the 255 a byte counter holds); 50 further vertices isolated
    n, R = leaves + 50, 32
    u = np.zeros(leaves, np.int32)
    v = np.arange(1, leaves + 1, dtype=np.int32)
    J = W.couplings_pm1(leaves, 3)
    lam = W.fields_normal(n, 0.2, 4)
    for orientation, (uu, vv) in ((0, (u, v)), (2, (v, u))):
        got, ref = run_graph_both(S, n, uu, vv, J, R, W.beta_grid(R, 0.1, 2.0, 8), 0.5, lam, 3,
                                  21, orientation=orientation)
        assert np.array_equal(got, ref), orientation


def test_graph_frozen_vertices_and_init_kinds(S):
    n, R = 400, 64
    u, v = W.erdos_renyi(n, 5.0, 8)
    J = W.couplings_pm1(u.size, 9)
    lam = W.fields_normal(n, 0.1, 10)
    frozen = np.zeros(n, np.uint8)
    frozen[::7] = 1
    for init in (0, 1, 2):
        got, ref = run_graph_both(S, n, u, v, J, R, 0.8, 1.0, lam, 3, 31, frozen=frozen,
                                  init=init)
        assert np.array_equal(got, ref), init
        assert np.all(got[:, frozen > 0] == 1)


@pytest.mark.parametrize("beta", [0.0, 1e-9, 40.0])
def test_graph_extreme_beta(S, beta):
    # beta = 0: T = 2^31 exactly for every class; beta = 40: nearly every T saturates
    n, R = 256, 32
    u, v = W.random_regular3(n, 5)
    J = W.couplings_pm1(u.size, 6)
    lam = W.fields_normal(n, 0.1, 7)
    got, ref = run_graph_both(S, n, u, v, J, R, beta, 1.0, lam, 3, 41)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("enc", ["INT8", "PACKED", "MULTISPIN"])
@pytest.mark.parametrize("beta,q,lam", [(0.0, 1.0, 0.0), (30.0, 0.3, 0.7), (2.0, 1e-6, -3.0)])
def test_lattice_extreme_parameters(S, enc, beta, q, lam):
    e = getattr(S, enc)
    L, R = (64, 32) if enc == "MULTISPIN" else (64, 1)
    mode = core.MODE_MULTISPIN if enc == "MULTISPIN" else core.MODE_SINGLE
    J, seed = 1.0, 51
    ctx = S.shaken_init(lattice_problem(S, e, L, R, beta, J, q, lam), seed)
    S.shaken_step(ctx, 3)
    S.shaken_step(ctx, 2)  # tiled path (fewer than 4 steps)
    got = S.shaken_get_spins(ctx, R, L * L).reshape(R, L, L)
    S.shaken_free(ctx)
    o = core.lattice_init(L, R, seed, mode, 0)
    o, _ = core.lattice_run(o, J, q, lam, beta, seed, 0, 5, mode)
    assert np.array_equal(got, o)


@pytest.mark.parametrize("init", [1, 2])
def test_lattice_init_kinds(S, init):
    L, R = 32, 32
    ctx = S.shaken_init(lattice_problem(S, S.MULTISPIN, L, R, 0.5, init=init), 3)
    s = S.shaken_get_spins(ctx, R, L * L)
    assert np.all(s == (1 if init == 1 else -1))
    S.shaken_step(ctx, 4)
    got = S.shaken_get_spins(ctx, R, L * L).reshape(R, L, L)
    S.shaken_free(ctx)
    o = (np.ones if init == 1 else lambda sh, dtype: -np.ones(sh, dtype))((R, L, L), np.int8)
    o, _ = core.lattice_run(o, 1.0, 1.0, 0.0, 0.5, 3, 0, 4, core.MODE_MULTISPIN)
    assert np.array_equal(got, o)


def test_set_spins_rejects_unfrozen_minus_on_frozen_site(S):
    L = 32
    fz = W.frozen_frame(L)
    ctx = S.shaken_init(lattice_problem(S, S.INT8, L, 1, 0.5, frozen=fz), 3)
    bad = -np.ones((1, L * L), np.int8)
    with pytest.raises(S.ShakenError):
        S.shaken_set_spins(ctx, bad)
    S.shaken_free(ctx)


def test_large_lattice_sampled(S):
    """INT8 L = 16384 (256 MiB per buffer): one full step, sampled sites against the
    oracle's single-site updates."""
    L, J, q, lam, beta, seed = 16384, 1.0, 1.0, 0.0, 0.44, 77
    ctx = S.shaken_init(lattice_problem(S, S.INT8, L, 1, beta, J, q, lam), seed)
    s0 = S.shaken_get_spins(ctx, 1, L * L).reshape(L, L)
    S.shaken_step(ctx, 1)
    s1 = S.shaken_get_spins(ctx, 1, L * L).reshape(L, L)
    S.shaken_free(ctx)
    g = np.random.default_rng(9)
    for _ in range(100):
        i, j = int(g.integers(L)), int(g.integers(L))
        sp = {}
        for (a, b) in ((i, j), ((i + 1) % L, j), (i, (j + 1) % L)):
            sp[(a, b)] = core.lattice_site(s0, a, b, J, q, lam, beta, seed, 0, 0,
                                           core.MODE_SINGLE, 0)
        saved = {k: s0[k] for k in sp}
        for k, val in sp.items():
            s0[k] = val
        tau = core.lattice_site(s0, i, j, J, q, lam, beta, seed, 0, 1, core.MODE_SINGLE, 0)
        for k, val in saved.items():
            s0[k] = val
        assert s1[i, j] == tau


@pytest.mark.parametrize("integer", [True, False])
def test_power_law_graph_with_hubs(S, integer):
    """Chung-Lu power-law graph (n = 20000, mean degree 6, exponent 2.5): a dozen
    vertices of degree above 255 (done by a whole warp), several hundred between 16
    and 255 (per-lane thresholds), the rest through the class tables; both
    orientations, so the hubs feed half 1 and then half 0.  Integer couplings:
    bit-exact against the oracle; real couplings: see the field-band tests (here the
    chain must only run and keep frozen vertices at +1)."""
    n, R = 20000, 64
    u, v = W.power_law(n, 6.0, 2.5, 3)
    J = W.couplings_pm1(u.size, 4) if integer else W.couplings_normal(u.size, 4)
    lam = W.fields_normal(n, 0.1, 5)
    frozen = np.zeros(n, np.uint8)
    frozen[1] = 1  # a hub
    for orientation, (uu, vv) in ((0, (u, v)), (2, (v, u))):
        if integer:
            got, ref = run_graph_both(S, n, uu, vv, J, R, 0.6, 1.0, lam, 2, 61,
                                      orientation=orientation, frozen=frozen)
            assert np.array_equal(got, ref), orientation
        else:
            ctx = S.shaken_init(graph_problem(S, n, uu, vv, J, R, 0.6, q=1.0, lam=lam,
                                              integer=False, orientation=orientation,
                                              frozen=frozen), 61)
            S.shaken_step(ctx, 3)
            got = S.shaken_get_spins(ctx, R, n)
            S.shaken_free(ctx)
            assert np.all(got[:, 1] == 1) and np.abs(got).min() == 1


@pytest.mark.parametrize("leaves", [1000, 100_000])
def test_star_hub_sampled(S, leaves):
    """A star with 10^3 or 10^5 leaves (centre 0, its degree far above what a byte
    counter holds) and +-1 couplings, oriented so the centre's 10^3 / 10^5 neighbours
    are its in-neighbours (half 0) and then its out-neighbours (half 1): every
    replica's decision at the centre in both half steps, and sampled leaves, against
    the oracle's single-vertex decisions (bit-plane draws, fp64 thresholds)."""
    n, R, q, beta, seed = leaves + 1, 64, 0.5, 0.004, 91
    hub_src = np.arange(1, n, dtype=np.int32)
    J = W.couplings_pm1(leaves, 7)
    lam = W.fields_normal(n, 0.2, 8)
    for uu, vv in ((hub_src, np.zeros(leaves, np.int32)), (np.zeros(leaves, np.int32), hub_src)):
        ctx = S.shaken_init(graph_problem(S, n, uu, vv, J, R, beta, q=q, lam=lam,
                                          orientation=S.ORIENT_GIVEN), seed)
        S.shaken_step(ctx, 1)
        s0 = S.shaken_get_spins(ctx, R, n)
        S.shaken_step(ctx, 1)
        sp = S.shaken_get_spins_prime(ctx, R, n)
        s1 = S.shaken_get_spins(ctx, R, n)
        S.shaken_free(ctx)
        tail, head = core.orient(uu, vv, 2)
        Jd, ld = J.astype(np.float64), lam.astype(np.float64)
        g = np.random.default_rng(5)
        for typ, src, out in ((0, s0, sp), (1, sp, s1)):
            inc = core.Incidence(n, tail, head, Jd, True, ld, q, typ)
            xs = [0] + [int(x) for x in g.integers(1, n, 40)]
            for x in xs:
                for r in (range(R) if x == 0 else g.integers(0, R, 4)):
                    tau = inc.site(src[int(r)], x, int(r), beta, seed, 1, core.DRAW_PLANE)
                    assert out[int(r), x] == tau, (typ, x, int(r))
