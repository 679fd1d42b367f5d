"""Pins of the exact small-system solver (oracle/exact.py) to the theorems of
arXiv:1904.06257 and to closed forms.  CPU only.

Each check is a statement the paper (or plain algebra) fixes independently of
the code: stochastic rows, Thm 2.1 (stationary measure, reversibility, marginal
of pi^b), the non-reversibility example after its proof, the identity
H(sigma, sigma) = H(sigma) - q|V| (Sec. 2 and Sec. 3), the lambda = 0 flip
symmetry, the ratio bound of Sec. 3.2, and the reduction of the lambda = 0
stationary measure to an anisotropic triangular Ising model.
"""
import itertools

import numpy as np
import pytest

from oracle import exact

L3 = 3
PARAMS = [  # (J, q, lam, beta)
    (1.0, 0.7, 0.3, 0.6),
    (1.0, 1.0, 0.0, 0.45),
    (-0.8, 0.4, -0.2, 1.1),
]


def lattice3(J, lam):
    tails, heads = exact.lattice_edges(L3)
    Jo = exact.oriented_matrix(L3 * L3, tails, heads, J)
    return exact.states(L3 * L3), tails, heads, Jo


@pytest.mark.parametrize("J,q,lam,beta", PARAMS)
def test_half_matrices_are_stochastic(J, q, lam, beta):
    S, t, h, Jo = lattice3(J, lam)
    for half in (0, 1):
        P = exact.half_matrix(S, Jo, lam, q, beta, half)
        assert np.allclose(P.sum(axis=1), 1.0, atol=1e-12)
        assert (P >= 0).all()


@pytest.mark.parametrize("J,q,lam,beta", PARAMS)
def test_thm21_stationary_and_reversible(J, q, lam, beta):
    S, t, h, Jo = lattice3(J, lam)
    P = exact.shaken_matrix(S, Jo, lam, q, beta)
    pi = exact.stationary(S, t, h, J, lam, q, beta)
    assert np.abs(pi @ P - pi).max() < 1e-14
    F = pi[:, None] * P
    assert np.abs(F - F.T).max() < 1e-15  # detailed balance (proof of Thm 2.1)
    # closed product form of Z->_sigma (includes the e^{beta sum lambda sigma} factor)
    pi2 = exact.stationary_product(S, Jo, lam, q, beta)
    assert np.abs(pi - pi2).max() < 1e-14
    # the lambda-free product misses stationarity whenever lambda != 0
    if lam != 0:
        hh = exact.fields(S, Jo, lam, q, 0)
        w = np.exp(np.logaddexp(beta * hh, -beta * hh).sum(axis=1))
        w /= w.sum()
        assert np.abs(w @ P - w).max() > 1e-6


def test_thm21_marginal_of_pair_gibbs_and_alt_dynamics():
    # small graph (4 vertices) so the pair space has 256 states
    tails = np.array([0, 1, 2, 0, 3])
    heads = np.array([1, 2, 3, 2, 1])
    J = np.array([1.0, -0.5, 0.8, 0.3, 1.2])
    lam = np.array([0.1, -0.2, 0.0, 0.25])
    q, beta = 0.6, 0.9
    S = exact.states(4)
    Jo = exact.oriented_matrix(4, tails, heads, J)
    pib = exact.pair_gibbs(S, tails, heads, J, lam, q, beta)
    pi = exact.stationary(S, tails, heads, J, lam, q, beta)
    N = S.shape[0]
    assert np.abs(pib.reshape(N, N).sum(axis=1) - pi).max() < 1e-14
    Palt = exact.alt_matrix(S, Jo, lam, q, beta)
    assert np.allclose(Palt.sum(axis=1), 1.0)
    assert np.abs(pib @ Palt - pib).max() < 1e-14
    # Eq. (eqshalt): summing P^alt over tau^(2) gives P^sh
    Psh = exact.shaken_matrix(S, Jo, lam, q, beta)
    red = Palt.reshape(N, N, N, N)[:, 0, :, :].sum(axis=2)
    assert np.abs(red - Psh).max() < 1e-14


def test_alt_dynamics_not_reversible_knn():
    # K_{2,2} with equal weights (the example after the proof of Thm 2.1):
    # sigma = (+1,+1) on every pair, tau = (+1,-1).
    n = 4  # vertices 0,1 | 2,3 ; edges between the parts
    tails = np.array([0, 0, 1, 1])
    heads = np.array([2, 3, 2, 3])
    J = np.ones(4)
    lam = np.zeros(4)
    q, beta = 0.5, 0.7
    S = exact.states(n)
    Jo = exact.oriented_matrix(n, tails, heads, J)
    pib = exact.pair_gibbs(S, tails, heads, J, lam, q, beta)
    Palt = exact.alt_matrix(S, Jo, lam, q, beta)
    N = S.shape[0]
    plus = exact.state_index(np.ones(n))
    minus = exact.state_index(-np.ones(n))
    a = plus * N + plus
    b = plus * N + minus
    lhs = pib[a] * Palt[a, b]
    rhs = pib[b] * Palt[b, a]
    assert abs(lhs - rhs) > 1e-6 * max(lhs, rhs)


@pytest.mark.parametrize("J,q,lam,beta", PARAMS)
def test_pair_energy_on_diagonal(J, q, lam, beta):
    S, t, h, Jo = lattice3(J, lam)
    Hs = exact.hamiltonian(S, t, h, J, lam)
    Hp = exact.pair_hamiltonian(S, S, t, h, J, lam, q)
    assert np.abs(Hp - (Hs - q * S.shape[1])).max() < 1e-12


def test_flip_symmetry_lambda0():
    S, t, h, Jo = lattice3(1.0, 0.0)
    P = exact.shaken_matrix(S, Jo, 0.0, 0.8, 0.5)
    flip = exact.state_index(-S)
    assert np.abs(P[np.ix_(flip, flip)] - P).max() < 1e-13


def test_ratio_bound_metastable_regime():
    # Sec. 3.2: for 0 < q < lambda < J, pi(sigma)/pi(+1) <= e^{-2 beta q} for sigma != +1
    J, q, lam, beta = 1.0, 0.1, 0.15, 2.0
    S, t, h, Jo = lattice3(J, lam)
    pi = exact.stationary(S, t, h, J, lam, q, beta)
    plus = exact.state_index(np.ones(9))
    ratio = np.delete(pi / pi[plus], plus)
    assert ratio.max() <= np.exp(-2 * beta * q) * (1 + 1e-12)


@pytest.mark.parametrize("J,q,beta", [(1.0, 0.5, 0.7), (1.0, 1.0, 0.45), (1.0, 2.0, 0.3)])
def test_lambda0_measure_is_anisotropic_triangular_gibbs(J, q, beta):
    S, t, h, Jo = lattice3(J, 0.0)
    pi = exact.stationary(S, t, h, J, 0.0, q, beta)
    tri = exact.triangular_gibbs_lambda0(S, L3, J, q, beta)
    assert np.abs(pi - tri).max() < 1e-14


def test_thm31_tv_to_gibbs_decreases_with_q():
    # Thm 3.1: with delta = e^{-2 beta q} small the shaken measure approaches Gibbs;
    # at fixed beta the TV distance falls as q grows (3x3 torus, exact).
    J, lam, beta = 1.0, 0.0, 0.4
    S, t, h, Jo = lattice3(J, lam)
    g = exact.gibbs(S, t, h, J, lam, beta)
    tv = [exact.total_variation(exact.stationary(S, t, h, J, lam, q, beta), g)
          for q in (0.5, 1.0, 2.0, 4.0, 8.0, 16.0)]
    assert all(a > b for a, b in zip(tv, tv[1:]))
    assert tv[-1] < 1e-4


def test_thm31_tv_trend_on_4x4_torus():
    """The same trend on a 4 x 4 torus (65,536 states), with pi in its product form
    (equal to Z->_sigma / Z, pinned on the 3 x 3 torus above): the TV distance to
    Gibbs falls strictly with q and is below 1e-5 at q = 16 (e^{-2 beta q} = 3e-6)."""
    J, lam, beta, L = 1.0, 0.0, 0.4, 4
    t, h = exact.lattice_edges(L)
    S = exact.states(L * L)
    Jo = exact.oriented_matrix(L * L, t, h, J)
    g = exact.gibbs(S, t, h, J, lam, beta)
    tv = [exact.total_variation(exact.stationary_product(S, Jo, lam, q, beta), g)
          for q in (0.5, 1.0, 2.0, 4.0, 8.0, 16.0)]
    assert all(a > b for a, b in zip(tv, tv[1:])), tv
    assert tv[-1] < 1e-5, tv


def test_frozen_set_restricts_chain():
    # a frozen site stays +1 and the restricted chain keeps Thm 2.1's measure
    J, q, lam, beta = 1.0, 0.6, 0.1, 0.8
    S, t, h, Jo = lattice3(J, lam)
    frozen = np.zeros(9, dtype=bool)
    frozen[[0, 4]] = True
    P = exact.shaken_matrix(S, Jo, lam, q, beta, frozen=frozen)
    ok = exact.allowed(S, frozen)
    assert np.allclose(P[ok].sum(axis=1), 1.0)
    pi = exact.stationary(S, t, h, J, lam, q, beta, frozen=frozen)
    assert np.abs(pi @ P - pi).max() < 1e-14
    F = pi[:, None] * P
    assert np.abs(F - F.T).max() < 1e-15


def test_reversed_order_same_measure():
    # Sec. 3: P^{sh'} (ur then dl) is the other composition; its stationary measure
    # is Z<- normalised, and both chains are reversible.
    J, q, lam, beta = 1.0, 0.7, 0.2, 0.6
    S, t, h, Jo = lattice3(J, lam)
    P2 = exact.shaken_matrix(S, Jo, lam, q, beta, order=(1, 0))
    w, v = np.linalg.eig(P2.T)
    k = np.argmin(np.abs(w - 1))
    pi2 = np.real(v[:, k])
    pi2 /= pi2.sum()
    F = pi2[:, None] * P2
    assert np.abs(F - F.T).max() < 1e-14


def test_generalised_split_is_reversible():
    # Sec. 5: J = J^o + J^oT with both orientations weighted; Thm 2.1 extends
    n = 5
    u = np.array([0, 1, 2, 3, 0, 1])
    v = np.array([1, 2, 3, 4, 4, 3])
    g = np.random.default_rng(4)
    J = g.standard_normal(6)
    lam = 0.2 * g.standard_normal(n)
    tails = np.concatenate([u, v])
    heads = np.concatenate([v, u])
    Jsplit = np.concatenate([0.3 * J, 0.7 * J])
    S = exact.states(n)
    Jo = exact.oriented_matrix(n, tails, heads, Jsplit)
    P = exact.shaken_matrix(S, Jo, lam, 0.9, 0.8)
    pi = exact.stationary(S, tails, heads, Jsplit, lam, 0.9, 0.8)
    assert np.abs(pi @ P - pi).max() < 1e-14
    F = pi[:, None] * P
    assert np.abs(F - F.T).max() < 1e-15
    # H(sigma, sigma) = H(sigma) - q|V| with H over the undirected couplings
    Hs = exact.hamiltonian(S, u, v, J, lam)
    Hp = exact.pair_hamiltonian(S, S, tails, heads, Jsplit, lam, 0.9)
    assert np.abs(Hp - (Hs - 0.9 * n)).max() < 1e-12


def test_triangular_critical_curve_reduces_to_square_at_q_equal_J():
    # Thm 4.1: 1 + tanh^3 J tanh q = 3 tanh J tanh q + 3 tanh^2 J; at q = J the
    # root is the square-lattice (Onsager) point tanh J = sqrt(2) - 1
    from scipy.optimize import brentq
    f = lambda x: 1 + np.tanh(x) ** 4 - 3 * np.tanh(x) ** 2 - 3 * np.tanh(x) ** 2
    Jc = brentq(f, 0.1, 1.0)
    assert abs(np.tanh(Jc) - (np.sqrt(2) - 1)) < 1e-12


# --------------------------------------------------------------------------- large-lattice references
def test_triangular_free_energy_reduces_to_onsager():
    # Kc = 0 is the square lattice: -(<ss>_a + <ss>_b) equals Onsager's closed form
    # (complete elliptic integral) on both sides of beta_c
    for b in (0.2, 0.35, 0.42, 0.46, 0.55, 0.8):
        ea, eb, _ = exact.triangular_bond_correlations(b, b, 0.0)
        assert abs(-(ea + eb) - exact.onsager_energy_per_site(b)) < 1e-8
    # anisotropic square lattice: the two correlations differ and swap with the couplings
    ea, eb, _ = exact.triangular_bond_correlations(0.3, 0.6, 0.0)
    eb2, ea2, _ = exact.triangular_bond_correlations(0.6, 0.3, 0.0)
    assert ea < eb and abs(ea - ea2) < 1e-10 and abs(eb - eb2) < 1e-10


def test_triangular_references_at_known_points():
    # isotropic triangular lattice at criticality (e^{4K} = 3): <ss> = 2/3 on every bond
    Kc = np.log(3.0) / 4.0
    for e in exact.triangular_bond_correlations(Kc, Kc, Kc):
        assert abs(e - 2.0 / 3.0) < 1e-6
    # high-temperature series: <ss>_a = t_a + 2 t_b t_c + O(t^3) (each bond lies in two
    # triangles), t = tanh K
    for K in (0.005, 0.01):
        ea, _, _ = exact.triangular_bond_correlations(K, 1.3 * K, 0.7 * K)
        ta, tb, tc = np.tanh(K), np.tanh(1.3 * K), np.tanh(0.7 * K)
        assert abs(ea - (ta + 2 * tb * tc)) < 10 * K ** 3


def test_triangular_magnetization_special_cases():
    # square lattice (Kc = 0): Onsager-Yang (1 - sinh^-4 2K)^(1/8), anisotropic form
    for Ka, Kb in ((0.45, 0.45), (0.5, 0.6), (0.7, 0.35)):
        ref = (1.0 - (np.sinh(2 * Ka) * np.sinh(2 * Kb)) ** -2) ** 0.125
        assert abs(exact.triangular_magnetization(Ka, Kb, 0.0) - ref) < 1e-12
    # isotropic triangular lattice (Potts): M^8 = 1 - 16 x^3 / ((1 + 3x)(1 - x)^3), x = e^{-4K}
    for K in (0.3, 0.35, 0.45):
        x = np.exp(-4 * K)
        ref = (1.0 - 16 * x ** 3 / ((1 + 3 * x) * (1 - x) ** 3)) ** 0.125
        assert abs(exact.triangular_magnetization(K, K, K) - ref) < 1e-12
    assert exact.triangular_magnetization(0.2, 0.2, 0.2) == 0.0  # disordered


def test_triangular_modulus_is_one_on_the_critical_surface():
    # criticality of the triangular model: sum over pairs sinh 2Ki sinh 2Kj = 1
    g = np.random.default_rng(4)
    for _ in range(20):
        a, b = g.uniform(0.05, 0.6, 2)
        sa, sb = np.sinh(2 * a), np.sinh(2 * b)
        sc = (1.0 - sa * sb) / (sa + sb)
        if sc <= 0:
            continue
        assert abs(exact.triangular_modulus(a, b, np.arcsinh(sc) / 2.0) - 1.0) < 1e-12


def test_shaken_critical_line_maps_to_triangular_criticality():
    # the honeycomb line tanh^2 K + 2 tanh K tanh Q = 1 of the doubling graph and the
    # triangular couplings (K1, K1, K2) of the lambda = 0 shaken measure give k = 1,
    # and beta_c tends to Onsager's 0.4407 as q grows (Thm 3.1)
    prev = None
    for q in (0.5, 1.0, 2.0, 4.0, 8.0, 16.0):
        bc = exact.shaken_lattice_beta_c(1.0, q)
        K1, K2 = exact.shaken_triangular_couplings(bc, 1.0, q)
        assert abs(exact.triangular_modulus(K1, K1, K2) - 1.0) < 1e-9
        if prev is not None:
            assert bc < prev
        prev = bc
    assert abs(prev - np.arctanh(np.sqrt(2.0) - 1.0)) < 1e-5


def test_shaken_equilibrium_matches_triangular_heat_bath():
    # the exact energy of the lambda = 0 shaken measure against an independent single-spin
    # heat bath of the same triangular model (paramagnetic point, 4 standard errors)
    beta, J, q = 0.45, 1.0, 1.0
    E_ref, m_ref = exact.shaken_lattice_equilibrium(beta, J, q)
    E, M = exact.triangular_heat_bath(48, J, q, beta, sweeps=600, burn=200, seed=3)
    se = exact.batch_means_se(E)
    assert m_ref == 0.0
    assert abs(E.mean() - E_ref) < 4 * se + 2e-3, (E.mean(), E_ref, se)
