"""Pins of the large-lattice references in oracle/exact.py (CPU)."""
import numpy as np

from oracle import exact


def test_onsager_energy_known_points():
    # at K_c = ln(1 + sqrt 2)/2 the energy per site is -sqrt(2)
    bc = 0.5 * np.log(1 + np.sqrt(2))
    assert abs(exact.onsager_energy_per_site(bc * (1 + 1e-7)) + np.sqrt(2)) < 1e-5
    # high-temperature series: u ~ -2 tanh K (1 + ...) ; at beta = 0.05: -2K - ... within 1e-3
    assert abs(exact.onsager_energy_per_site(0.05) + 2 * np.tanh(0.05)) < 2e-3
    # ground state
    assert abs(exact.onsager_energy_per_site(5.0) + 2.0) < 1e-8


def test_triangular_heat_bath_matches_exact_small_lattice():
    # 3x3 torus: the heat bath's energy average equals the exact shaken stationary average
    L, J, q, beta = 3, 1.0, 0.8, 0.5
    tails, heads = exact.lattice_edges(L)
    S = exact.states(L * L)
    pi = exact.stationary(S, tails, heads, J, 0.0, q, beta)
    E = exact.hamiltonian(S, tails, heads, J, 0.0) / (L * L)
    ref = float(pi @ E)
    samples, _ = exact.triangular_heat_bath(L, J, q, beta, sweeps=40000, burn=200, seed=3)
    se = exact.batch_means_se(samples)
    assert abs(samples.mean() - ref) < 5 * se + 1e-9


def _oracle_m(L, R, q, lam, beta, seed, burn, blocks, every):
    """Per-replica time average of m = sum sigma / |V| over `blocks` samples taken
    every `every` full steps after `burn` steps, oracle chain from a random start."""
    from oracle import core
    s = core.lattice_init(L, R, seed, core.MODE_SINGLE)
    s, _ = core.lattice_run(s, 1.0, q, lam, beta, seed, 0, burn, core.MODE_SINGLE)
    ms = []
    for k in range(blocks):
        s, _ = core.lattice_run(s, 1.0, q, lam, beta, seed, burn + every * k, every,
                                core.MODE_SINGLE)
        ms.append(s.reshape(R, -1).mean(axis=1))
    return np.mean(ms, axis=0)


def test_small_field_orders_the_magnetisation():
    """lambda = 0.01 has no closed form at finite size; the sign and the ordering
    are fixed: m(-0.01) < m(0) < m(0.01) at equal beta and q (the field term
    lambda sigma of Eq. ham1 favours +1).  The same seed for the three runs makes
    the differences sharp; each must exceed 4 standard errors over 32 replicas."""
    L, R, q, beta, seed = 16, 32, 1.0, 0.4407, 0x5348414B
    m = {lam: _oracle_m(L, R, q, lam, beta, seed, 50, 15, 6) for lam in (-0.01, 0.0, 0.01)}
    for lo, hi in ((-0.01, 0.0), (0.0, 0.01)):
        d = m[hi] - m[lo]
        assert d.mean() > 4 * d.std(ddof=1) / np.sqrt(R), (lo, hi, d.mean())


def test_small_field_exact_mean_is_increasing_and_odd():
    """The same ordering under the exact stationary measure of a 3 x 3 torus
    (closed-form pi with its e^{beta sum lambda sigma} factor), and the flip
    symmetry m(-lambda) = -m(lambda)."""
    L, J, q, beta = 3, 1.0, 1.0, 0.4407
    tails, heads = exact.lattice_edges(L)
    S = exact.states(L * L)
    M = S.sum(axis=1) / (L * L)
    mean = {}
    for lam in (-0.01, 0.0, 0.01):
        pi = exact.stationary(S, tails, heads, J, lam, q, beta)
        mean[lam] = float(pi @ M)
    assert mean[-0.01] < mean[0.0] < mean[0.01]
    assert abs(mean[0.0]) < 1e-12 and abs(mean[0.01] + mean[-0.01]) < 1e-12
