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
