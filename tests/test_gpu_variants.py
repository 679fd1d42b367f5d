"""Variants of the shaken dynamics on the GPU path:
* the reversed order P^{sh'} = P^ur then P^dl (Sec. 3), bit-exact against the
  oracle applying the two half steps in that order;
* the generalised dynamics of Sec. 5 (J = J^o + J^oT, both orientations weighted;
  J^o = J/2 is the symmetric PCA), fed as an oriented edge list: the GPU chain's
  law against the exact transition matrix (chi-square);
* the triangular lattice of Sec. 4 (three right / three left neighbours) through
  the graph path, bit-exact against the oracle; at q = J its pair (sigma, sigma')
  is the square-lattice Ising model (Thm 4.1 and the figure of Sec. 4), so the pair
  energy per site and |m| follow Onsager on both sides of beta_c = 0.4407."""
import numpy as np
import pytest
from scipy import stats

from oracle import core, exact
from paper_1904_06257_gb300 import workloads as W
from tests.gpu_util import graph_problem, lattice_problem, lib, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    require_cuda()
    return lib()


@pytest.mark.parametrize("enc,L,R,steps", [("INT8", 64, 2, 5), ("PACKED", 96, 1, 2),
                                           ("MULTISPIN", 32, 32, 6), ("MULTISPIN", 96, 32, 3)])
def test_reversed_order_lattice(S, enc, L, R, steps):
    e = getattr(S, enc)
    mode = core.MODE_MULTISPIN if enc == "MULTISPIN" else core.MODE_SINGLE
    J, q, lam, seed = 1.0, 0.7, 0.05, 123
    beta = W.beta_grid(R, 0.3, 0.6, 5)
    ctx = S.shaken_init(lattice_problem(S, e, L, R, beta, J, q, lam), seed)
    S.shaken_set_order(ctx, True)
    S.shaken_step(ctx, steps)
    got = S.shaken_get_spins(ctx, R, L * L).reshape(R, L, L)
    S.shaken_free(ctx)
    o = core.lattice_init(L, R, seed, mode, 0)
    for t in range(steps):
        sp = core.lattice_half(o, J, q, lam, beta, seed, t, 1, mode)  # ur first
        o = core.lattice_half(sp, J, q, lam, beta, seed, t, 0, mode)
    assert np.array_equal(got, o)


def test_reversed_order_graph(S):
    n, R = 500, 32
    u, v = W.erdos_renyi(n, 6.0, 3)
    J = W.couplings_pm1(u.size, 4)
    lam = W.fields_normal(n, 0.1, 5)
    seed = 77
    ctx = S.shaken_init(graph_problem(S, n, u, v, J, R, 0.9, q=1.0, lam=lam), seed)
    S.shaken_set_order(ctx, True)
    S.shaken_step(ctx, 4)
    got = S.shaken_get_spins(ctx, R, n)
    S.shaken_free(ctx)
    tail, head = core.orient(u, v, 0)
    o = core.graph_init(n, R, seed, 0)
    for t in range(4):
        sp = core.graph_half(o, tail, head, J.astype(np.float64), True, lam.astype(np.float64),
                             1.0, 0.9, seed, t, 1, draw=core.DRAW_PLANE)
        o = core.graph_half(sp, tail, head, J.astype(np.float64), True, lam.astype(np.float64),
                            1.0, 0.9, seed, t, 0, draw=core.DRAW_PLANE)
    assert np.array_equal(got, o)


def _chi2_pvalue(counts, probs, nrep):
    exp_ = probs * nrep
    big = exp_ >= 5
    obs = np.append(counts[big], counts[~big].sum())
    ex = np.append(exp_[big], exp_[~big].sum())
    if ex[-1] == 0:
        obs, ex = obs[:-1], ex[:-1]
    return stats.chisquare(obs, ex * obs.sum() / ex.sum()).pvalue


@pytest.mark.parametrize("frac", [0.5, 0.25])
def test_generalised_split_follows_exact_law(S, frac):
    n, R = 6, 32 * 256
    u = np.array([0, 1, 2, 3, 4, 5, 0, 2], dtype=np.int32)
    v = np.array([1, 2, 3, 4, 5, 0, 3, 5], dtype=np.int32)
    g = np.random.default_rng(2)
    J = g.standard_normal(8).astype(np.float32)
    lam = (0.3 * g.standard_normal(n)).astype(np.float32)
    uu, vv, JJ = W.split_both_ways(u, v, J, frac)
    q, beta = 0.8, 0.7
    s0 = np.array([1, -1, 1, 1, -1, -1], dtype=np.int8)
    Sx = exact.states(n)
    Jo = exact.oriented_matrix(n, uu, vv, JJ.astype(np.float64))
    P = exact.shaken_matrix(Sx, Jo, lam.astype(np.float64), q, beta)
    mu0 = np.zeros(Sx.shape[0])
    mu0[exact.state_index(s0)] = 1.0
    for t in (1, 2):
        init = np.broadcast_to(s0, (R, n)).copy()
        ctx = S.shaken_init(graph_problem(S, n, uu, vv, JJ, R, beta, q=q, lam=lam, integer=False,
                                          orientation=S.ORIENT_GIVEN, init=S.INIT_GIVEN,
                                          init_spins=init), 1000 + t)
        S.shaken_step(ctx, t)
        st = S.shaken_get_spins(ctx, R, n)
        S.shaken_free(ctx)
        counts = np.bincount(exact.state_index(st), minlength=Sx.shape[0]).astype(float)
        assert _chi2_pvalue(counts, exact.evolve(mu0, P, t), R) > 1e-4


def test_triangular_lattice_bit_exact(S):
    L, R = 12, 64
    u, v = W.triangular_lattice_as_graph(L)
    J = np.ones(u.size, dtype=np.float32)
    seed = 5
    ctx = S.shaken_init(graph_problem(S, L * L, u, v, J, R, W.beta_grid(R, 0.1, 0.6, 16), q=0.6,
                                      lam_c=0.0, orientation=S.ORIENT_GIVEN), seed)
    S.shaken_step(ctx, 5)
    got = S.shaken_get_spins(ctx, R, L * L)
    S.shaken_free(ctx)
    tail, head = core.orient(u, v, 2)
    o = core.graph_init(L * L, R, seed, 0)
    o, _ = core.graph_run(o, tail, head, J.astype(np.float64), True, 0.0, 0.6,
                          W.beta_grid(R, 0.1, 0.6, 16), seed, 0, 5, draw=core.DRAW_PLANE)
    assert np.array_equal(got, o)


@pytest.mark.parametrize("beta", [0.35, 0.48])
def test_triangular_at_q_equal_J_follows_onsager(S, beta):
    """Triangular lattice, J = q = 1, lambda = 0: the pair Hamiltonian lives on a
    square lattice of 2 L^2 sites, so the stationary pair energy per site is Onsager's
    u(beta) and, in the ordered phase (beta = 0.48 > 0.4407), E|m| is the spontaneous
    magnetisation (1 - sinh^-4(2 beta))^(1/8) = 0.8775.  64 replicas of a 96 x 96
    torus; finite-size corrections are exponentially small this far from beta_c."""
    L, R = 96, 64
    u, v = W.triangular_lattice_as_graph(L)
    J = np.ones(u.size, dtype=np.float32)
    ctx = S.shaken_init(graph_problem(S, L * L, u, v, J, R, beta, q=1.0, lam_c=0.0,
                                      orientation=S.ORIENT_GIVEN, init=1), 77)
    S.shaken_step(ctx, 300)
    e, m = [], []
    for _ in range(40):
        S.shaken_step(ctx, 10)
        o = S.shaken_observables(ctx, R)
        e.append(o["pair_energy"] / (2 * L * L))
        m.append(np.abs(o["magnetization"]))
    S.shaken_free(ctx)
    e, m = np.array(e).mean(axis=0), np.array(m).mean(axis=0)  # per replica
    u_ref = exact.onsager_energy_per_site(beta)
    se = e.std(ddof=1) / np.sqrt(R)
    assert abs(e.mean() - u_ref) < 4 * se + 2e-3, (e.mean(), u_ref, se)
    if beta > 0.4407:
        m_ref = (1.0 - np.sinh(2 * beta) ** -4) ** 0.125
        sem = m.std(ddof=1) / np.sqrt(R)
        assert abs(m.mean() - m_ref) < 4 * sem + 5e-3, (m.mean(), m_ref, sem)
    else:
        assert m.mean() < 0.05


def _thm41_beta_c(q_over_J):
    """Root in beta of the critical curve of Thm 4.1 for the triangular shaken
    dynamics, 1 + tanh^3(bJ) tanh(bq) = 3 tanh(bJ) tanh(bq) + 3 tanh^2(bJ), J = 1."""
    from scipy.optimize import brentq

    def f(b):
        tJ, tq = np.tanh(b), np.tanh(q_over_J * b)
        return 1.0 + tJ ** 3 * tq - 3.0 * tJ * tq - 3.0 * tJ ** 2

    return brentq(f, 0.05, 5.0)


def _binder(S, L, q, beta, R, seed, burn=3000, meas=6000, chunk=1000):
    """Binder cumulant U4 = 1 - <m^4> / (3 <m^2>^2) of the full-step configurations of
    the triangular shaken chain (J = 1, lambda = 0) on an L x L torus, R independent
    replicas from +1, and its standard error by the jackknife over replicas (the
    replicas are independent; each contributes its time averages)."""
    u, v = W.triangular_lattice_as_graph(L)
    J = np.ones(u.size, dtype=np.float32)
    ctx = S.shaken_init(graph_problem(S, L * L, u, v, J, R, beta, q=q, lam_c=0.0,
                                      orientation=S.ORIENT_GIVEN, init=1), seed)
    S.shaken_step(ctx, burn)
    m2 = np.zeros(R)
    m4 = np.zeros(R)
    for _ in range(meas // chunk):
        m, _ = S.shaken_step_record(ctx, chunk, R)
        m2 += (m ** 2).sum(axis=0)
        m4 += (m ** 4).sum(axis=0)
    S.shaken_free(ctx)
    m2 /= meas
    m4 /= meas
    u4 = 1.0 - m4.mean() / (3.0 * m2.mean() ** 2)
    tot2, tot4 = m2.sum(), m4.sum()
    jk = 1.0 - ((tot4 - m4) / (R - 1)) / (3.0 * ((tot2 - m2) / (R - 1)) ** 2)
    se = np.sqrt((R - 1) / R * ((jk - jk.mean()) ** 2).sum())
    return u4, se


@pytest.mark.parametrize("q", [0.5, 2.0])
def test_triangular_critical_curve_binder_crossing(S, q):
    """Thm 4.1 away from q = J: the Binder cumulants of the triangular shaken chain on
    24 x 24 and 48 x 48 tori cross at the root beta_c of the critical curve.  Below
    beta_c (0.95 beta_c) the larger lattice has the smaller U4 (disordered), above it
    (1.05 beta_c) the larger one (ordered), each by more than 3 standard errors; the
    q = J point (0.4407), which the curve gives only for q = J, lies outside that
    window for both q.  Linear interpolation of the difference puts the crossing
    within 2% of beta_c."""
    bc = _thm41_beta_c(q)
    assert abs(bc / 0.44068679350977 - 1.0) > 0.1  # the curve really moves with q
    R = 2048
    rows = []
    for k, f in enumerate((0.95, 1.0, 1.05)):
        beta = f * bc
        u_s, e_s = _binder(S, 24, q, beta, R, 100 + k)
        u_l, e_l = _binder(S, 48, q, beta, R, 200 + k)
        rows.append((beta, u_l - u_s, np.hypot(e_s, e_l), u_s, u_l))
    print("beta_c", bc, [tuple(round(float(x), 4) for x in r) for r in rows])
    (b0, d0, s0, *_), (b1, d1, s1, *_), (b2, d2, s2, *_) = rows
    assert d0 < -3 * s0 and d2 > 3 * s2, rows
    # crossing by linear interpolation on the bracketing pair
    if d1 < 0:
        cross = b1 + (b2 - b1) * (-d1) / (d2 - d1)
    else:
        cross = b0 + (b1 - b0) * (-d0) / (d1 - d0)
    assert abs(cross / bc - 1.0) < 0.02, (cross, bc, rows)
