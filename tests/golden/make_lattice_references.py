"""Write lattice_references.json: exact stationary values of the lattice shaken chain
at lambda = 0 for the plain-lattice sweep (L = 4096; q in {0.5, 1, 2, 4, 8, 16},
beta in {0.40, 0.4407, 0.48}, J = 1), computed by oracle/exact.py only.

At lambda = 0 the stationary measure of the shaken chain on the square lattice is
the Gibbs measure of an anisotropic triangular Ising model (couplings K1 on the two
square bonds, K2 on one diagonal; summing out the second copy of the doubling graph,
Thm 2.1 and Sec. 3).  Its energy per site H(sigma)/|V| = -J (<s s>_down + <s s>_left)
comes from Houtappel's free energy, |m| from the elliptic modulus k, and beta_c from
the hexagonal doubling graph's critical line.  Run: python tests/golden/make_lattice_references.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact  # noqa: E402

QS = (0.5, 1.0, 2.0, 4.0, 8.0, 16.0)
BETAS = (0.40, 0.4407, 0.48)


def main():
    rows = []
    for q in QS:
        bc = exact.shaken_lattice_beta_c(1.0, q)
        for beta in BETAS:
            e, m = exact.shaken_lattice_equilibrium(beta, 1.0, q)
            K1, K2 = exact.shaken_triangular_couplings(beta, 1.0, q)
            rows.append({"q": q, "beta": beta, "J": 1.0, "lambda": 0.0, "beta_c": bc,
                         "energy_per_site": e, "abs_m": m, "K1": K1, "K2": K2})
    onsager = {str(b): exact.onsager_energy_per_site(b) for b in BETAS}
    out = {"source": "oracle/exact.py (Houtappel free energy, elliptic modulus, honeycomb "
                     "critical line); see make_lattice_references.py",
           "points": rows, "onsager_energy_per_site": onsager}
    with open(os.path.join(HERE, "lattice_references.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
