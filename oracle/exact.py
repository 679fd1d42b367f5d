"""Exact small-system solver for the shaken dynamics (numpy, fp64).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

Everything here is a direct transcription of a definition of arXiv:1904.06257
on the full configuration space {-1,+1}^V (|V| <= ~12):

* ``hamiltonian``       -- H(sigma), Eq. (ham1): -sum_{e} J_e s_x s_y - 2 sum_x lambda_x s_x.
* ``pair_hamiltonian``  -- H(sigma1, sigma2), Eq. (ham21).
* ``half_matrix``       -- P^{1->2} / P^{2->1} as products of single-site heat-bath
                           factors e^{beta h tau} / 2cosh(beta h), Sec. 2 (and the
                           lattice P^{dl}, P^{ur} of Sec. 3).
* ``z_forward``         -- Z->_sigma = sum_tau e^{-beta H(sigma, tau)}, Thm 2.1.
* ``stationary``        -- pi(sigma) = Z->_sigma / Z, Thm 2.1.
* ``alt_matrix``        -- P^{alt} on pairs, Eq. (Palt), and ``pair_gibbs`` pi^b, Eq. (pi2).
* ``gibbs``             -- pi^G(sigma) ~ e^{-beta H(sigma)}, Eq. (piG).

A graph is given by its oriented edge list E^o (tail -> head) and couplings;
the doubling graph of Def. 2.1 joins tail^(1) to head^(2).  Frozen sites
(Sec. 3, the set B) restrict the configuration space to sigma_x = +1 on B.
"""
from __future__ import annotations

import itertools

import numpy as np


def states(n: int) -> np.ndarray:
    """All configurations of n spins, shape (2^n, n); state i has sigma_x = +1 iff bit x of i."""
    idx = np.arange(1 << n, dtype=np.int64)
    bits = (idx[:, None] >> np.arange(n)[None, :]) & 1
    return (2 * bits - 1).astype(np.int64)


def state_index(sig: np.ndarray) -> np.ndarray:
    """Inverse of ``states``: configurations (..., n) -> integer index."""
    sig = np.asarray(sig)
    bits = (sig > 0).astype(np.int64)
    return (bits << np.arange(sig.shape[-1])).sum(axis=-1)


def lattice_edges(L: int):
    """Oriented lattice edges (x -> x_up), (x -> x_right) on the L x L torus (Sec. 3,
    Eq. (ham2)); x = (i, j) -> i*L + j, up = row i+1, right = column j+1."""
    tails, heads = [], []
    for i in range(L):
        for j in range(L):
            x = i * L + j
            tails += [x, x]
            heads += [((i + 1) % L) * L + j, i * L + (j + 1) % L]
    return np.array(tails), np.array(heads)


def oriented_matrix(n, tails, heads, J):
    """J^o with J^o[tail, head] = J_e (duplicate edges add), Sec. 2 (matrix form)."""
    Jo = np.zeros((n, n))
    np.add.at(Jo, (np.asarray(tails), np.asarray(heads)), np.broadcast_to(J, np.shape(tails)))
    return Jo


def fields(S, Jo, lam, q, half):
    """Local fields for every configuration (rows of S).
    half 0: h^{1->2}(sigma) = J^{oT} sigma + q sigma + lambda;
    half 1: h^{2->1}(sigma) = J^o sigma + q sigma + lambda   (Sec. 2)."""
    lam = np.broadcast_to(np.asarray(lam, dtype=float), (S.shape[1],))
    if half == 0:
        coup = S @ Jo  # (J^{oT} sigma)_x = sum_y Jo[y, x] sigma_y
    else:
        coup = S @ Jo.T  # (J^o sigma)_x = sum_y Jo[x, y] sigma_y
    return coup + q * S + lam[None, :]


def allowed(S, frozen):
    if frozen is None:
        return np.ones(S.shape[0], dtype=bool)
    f = np.asarray(frozen, dtype=bool)
    return np.all(S[:, f] > 0, axis=1)


def half_matrix(S, Jo, lam, q, beta, half, frozen=None):
    """P[sigma, tau] = prod_{x not in B} e^{beta h_x(sigma) tau_x} / 2cosh(beta h_x(sigma)),
    restricted to configurations with +1 on B (zero rows/columns elsewhere)."""
    h = fields(S, Jo, lam, q, half)
    free = np.ones(S.shape[1], dtype=bool) if frozen is None else ~np.asarray(frozen, dtype=bool)
    bh = beta * h[:, free]
    logZ = np.logaddexp(bh, -bh).sum(axis=1)  # sum_x log 2cosh(beta h_x)
    logP = bh @ S[:, free].T - logZ[:, None]
    P = np.exp(logP)
    ok = allowed(S, frozen)
    P[~ok, :] = 0.0
    P[:, ~ok] = 0.0
    return P


def shaken_matrix(S, Jo, lam, q, beta, frozen=None, order=(0, 1)):
    """P^{sh} = P^{1->2} P^{2->1} (Sec. 2); order=(1, 0) gives P^{sh'} (Sec. 3)."""
    A = half_matrix(S, Jo, lam, q, beta, order[0], frozen)
    B = half_matrix(S, Jo, lam, q, beta, order[1], frozen)
    return A @ B


def hamiltonian(S, tails, heads, J, lam):
    """H(sigma) = -sum_{e} J_e s_tail s_head - 2 sum_x lambda_x s_x, Eq. (ham1)."""
    S = np.atleast_2d(S)
    lam = np.broadcast_to(np.asarray(lam, dtype=float), (S.shape[1],))
    J = np.broadcast_to(np.asarray(J, dtype=float), np.shape(tails))
    return -(S[:, tails] * S[:, heads] * J).sum(axis=1) - 2.0 * (S * lam).sum(axis=1)


def pair_hamiltonian(S1, S2, tails, heads, J, lam, q):
    """H(s1, s2) = -sum_{(x,y) in E^o} J s1_x s2_y - sum_x (q s1_x s2_x + lambda_x (s1_x + s2_x)),
    Eq. (ham21)."""
    S1 = np.atleast_2d(S1)
    S2 = np.atleast_2d(S2)
    lam = np.broadcast_to(np.asarray(lam, dtype=float), (S1.shape[1],))
    J = np.broadcast_to(np.asarray(J, dtype=float), np.shape(tails))
    return (-(S1[:, tails] * S2[:, heads] * J).sum(axis=1)
            - (q * S1 * S2 + lam * (S1 + S2)).sum(axis=1))


def z_forward(S, tails, heads, J, lam, q, beta, frozen=None):
    """Z->_sigma = sum_{tau allowed} e^{-beta H(sigma, tau)} by brute force (Thm 2.1)."""
    ok = allowed(S, frozen)
    T = S[ok]
    out = np.zeros(S.shape[0])
    for a in range(S.shape[0]):
        H = pair_hamiltonian(np.repeat(S[a:a + 1], T.shape[0], 0), T, tails, heads, J, lam, q)
        out[a] = np.exp(-beta * H).sum()
    out[~ok] = 0.0
    return out


def stationary(S, tails, heads, J, lam, q, beta, frozen=None):
    """pi(sigma) = Z->_sigma / Z, Thm 2.1 (Eq. (mispi))."""
    z = z_forward(S, tails, heads, J, lam, q, beta, frozen)
    return z / z.sum()


def stationary_product(S, Jo, lam, q, beta, frozen=None):
    """The same measure written as a product over sites (no frozen sites):
    pi(sigma) ~ exp(beta sum_x lambda_x sigma_x) prod_x 2cosh(beta h^{1->2}_x(sigma))."""
    assert frozen is None
    lam_v = np.broadcast_to(np.asarray(lam, dtype=float), (S.shape[1],))
    h = fields(S, Jo, lam, q, 0)
    logw = beta * (S * lam_v).sum(axis=1) + np.logaddexp(beta * h, -beta * h).sum(axis=1)
    w = np.exp(logw - logw.max())
    return w / w.sum()


def gibbs(S, tails, heads, J, lam, beta, frozen=None):
    """pi^G(sigma) = e^{-beta H(sigma)} / Z^G, Eq. (piG)."""
    H = hamiltonian(S, tails, heads, J, lam)
    w = np.exp(-beta * (H - H.min()))
    w[~allowed(S, frozen)] = 0.0
    return w / w.sum()


def pair_gibbs(S, tails, heads, J, lam, q, beta):
    """pi^b(s1, s2) = e^{-beta H(s1, s2)} / Z on pairs (index a*2^n + b), Eq. (pi2)."""
    N = S.shape[0]
    a, b = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    H = pair_hamiltonian(S[a.ravel()], S[b.ravel()], tails, heads, J, lam, q)
    w = np.exp(-beta * (H - H.min()))
    return w / w.sum()


def alt_matrix(S, Jo, lam, q, beta):
    """P^{alt}((s1, s2), (t1, t2)) = P^{1->2}(s1, t2) P^{2->1}(t2, t1), Eq. (Palt).
    Pair states are indexed a*2^n + b for (s1 = S[a], s2 = S[b])."""
    A = half_matrix(S, Jo, lam, q, beta, 0)
    B = half_matrix(S, Jo, lam, q, beta, 1)
    N = S.shape[0]
    P = np.zeros((N * N, N * N))
    for a1 in range(N):
        for t1 in range(N):
            # independent of s2: same row for every b1
            row = A[a1, :] * B[:, t1]  # indexed by t2
            for b1 in range(N):
                P[a1 * N + b1, t1 * N + np.arange(N)] = row
    return P


def total_variation(mu, nu):
    """||mu - nu||_TV = (1/2) sum |mu - nu|, Eq. (dist)."""
    return 0.5 * np.abs(np.asarray(mu) - np.asarray(nu)).sum()


def evolve(mu0, P, t):
    mu = np.asarray(mu0, dtype=float)
    for _ in range(t):
        mu = mu @ P
    return mu


def triangular_gibbs_lambda0(S, L, J, q, beta):
    """Gibbs measure of the anisotropic triangular Ising model obtained from the
    shaken measure at lambda = 0 by summing out the second copy: couplings
    K1 on (x, x_down) and (x, x_left), K2 on (x_down, x_left), with K = beta J,
    Q = beta q:  K1 = (1/4) ln[cosh(2K+Q)/cosh(2K-Q)],
    K2 = (1/4) ln[cosh(2K+Q) cosh(2K-Q)/cosh^2 Q]."""
    K, Q = beta * J, beta * q
    K1 = 0.25 * np.log(np.cosh(2 * K + Q) / np.cosh(2 * K - Q))
    K2 = 0.25 * np.log(np.cosh(2 * K + Q) * np.cosh(2 * K - Q) / np.cosh(Q) ** 2)
    logw = np.zeros(S.shape[0])
    for i, j in itertools.product(range(L), range(L)):
        x = i * L + j
        dn = ((i - 1) % L) * L + j
        lf = i * L + (j - 1) % L
        logw += K1 * S[:, x] * (S[:, dn] + S[:, lf]) + K2 * S[:, dn] * S[:, lf]
    w = np.exp(logw - logw.max())
    return w / w.sum()


# ----------------------------------------------------------------------------- large lattices
def onsager_energy_per_site(beta: float, J: float = 1.0) -> float:
    """Energy per site of the square-lattice Ising model (Onsager):
    u = -J coth(2K) [1 + (2/pi) (2 tanh^2(2K) - 1) K(k)],  k = 2 sinh(2K) / cosh^2(2K),
    K the complete elliptic integral of the first kind (argument m = k^2)."""
    from scipy.special import ellipk
    K = beta * J
    k = 2.0 * np.sinh(2 * K) / np.cosh(2 * K) ** 2
    return -J / np.tanh(2 * K) * (1.0 + (2.0 / np.pi) * (2.0 * np.tanh(2 * K) ** 2 - 1.0)
                                  * ellipk(k * k))


def shaken_triangular_couplings(beta: float, J: float, q: float):
    """(K1, K2) of the anisotropic triangular Ising model that the lambda = 0 shaken
    measure on the square lattice equals (see ``triangular_gibbs_lambda0``)."""
    K, Q = beta * J, beta * q
    K1 = 0.25 * np.log(np.cosh(2 * K + Q) / np.cosh(2 * K - Q))
    K2 = 0.25 * np.log(np.cosh(2 * K + Q) * np.cosh(2 * K - Q) / np.cosh(Q) ** 2)
    return K1, K2


def triangular_free_energy(Ka: float, Kb: float, Kc: float, n: int = 1 << 15) -> float:
    """-beta f per site of the Ising model on the triangular lattice with couplings
    Ka, Kb, Kc on its three bond directions (one bond of each per site), Houtappel's
    solution: -beta f = ln 2 + (1/8 pi^2) int int ln D(t1, t2) dt1 dt2 over [0, 2 pi]^2,
    D = ca cb cc + sa sb sc - sa cos t1 - sb cos t2 - sc cos(t1 + t2), c = cosh 2K,
    s = sinh 2K.  For fixed t1, D = A - R cos(t2 - phi) with A = ca cb cc + sa sb sc -
    sa cos t1 and R^2 = sb^2 + sc^2 + 2 sb sc cos t1, and the t2 integral is
    2 pi ln[(A + sqrt(A^2 - R^2)) / 2]; the remaining t1 integral of a smooth periodic
    function is taken by the midpoint rule on n points.  Kc = 0 is Onsager's square
    lattice."""
    ca, cb, cc = np.cosh(2 * Ka), np.cosh(2 * Kb), np.cosh(2 * Kc)
    sa, sb, sc = np.sinh(2 * Ka), np.sinh(2 * Kb), np.sinh(2 * Kc)
    t = (np.arange(n) + 0.5) * (2.0 * np.pi / n)
    A = ca * cb * cc + sa * sb * sc - sa * np.cos(t)
    R2 = sb * sb + sc * sc + 2.0 * sb * sc * np.cos(t)
    g = np.log(0.5 * (A + np.sqrt(np.maximum(A * A - R2, 0.0))))
    return float(np.log(2.0) + 0.5 * g.mean())


def triangular_bond_correlations(Ka: float, Kb: float, Kc: float, h: float = 1e-5):
    """Nearest-neighbour correlations <s s> on the three bond directions,
    d(-beta f)/dK_a, by central differences of ``triangular_free_energy``."""
    out = []
    for d in ((h, 0, 0), (0, h, 0), (0, 0, h)):
        fp = triangular_free_energy(Ka + d[0], Kb + d[1], Kc + d[2])
        fm = triangular_free_energy(Ka - d[0], Kb - d[1], Kc - d[2])
        out.append((fp - fm) / (2.0 * h))
    return tuple(out)


def triangular_modulus(Ka: float, Kb: float, Kc: float) -> float:
    """Elliptic modulus k of the ferromagnetic triangular Ising model with couplings
    Ka, Kb, Kc (v = tanh K):
    k = (1 - va^2)(1 - vb^2)(1 - vc^2) / (4 sqrt[(1 + va vb vc)(va + vb vc)(vb + va vc)(vc + va vb)]);
    k = 1 at criticality, k < 1 in the ordered phase.  Kc = 0 gives the square
    lattice's k = 1 / (sinh 2Ka sinh 2Kb)."""
    va, vb, vc = np.tanh(Ka), np.tanh(Kb), np.tanh(Kc)
    num = (1 - va * va) * (1 - vb * vb) * (1 - vc * vc)
    den = 4.0 * np.sqrt((1 + va * vb * vc) * (va + vb * vc) * (vb + va * vc) * (vc + va * vb))
    return float(num / den)


def triangular_magnetization(Ka: float, Kb: float, Kc: float) -> float:
    """Spontaneous magnetisation (1 - k^2)^(1/8) in the ordered phase (k < 1), else 0."""
    k = triangular_modulus(Ka, Kb, Kc)
    return float((1.0 - k * k) ** 0.125) if k < 1.0 else 0.0


def shaken_lattice_equilibrium(beta: float, J: float, q: float):
    """Stationary energy per site H(sigma)/|V| = -J (<s_x s_down> + <s_x s_left>) and
    spontaneous |m| of the lattice shaken chain at lambda = 0, from the exact
    anisotropic triangular Gibbs measure it equals (reading of Sec. 3, Thm 2.1)."""
    K1, K2 = shaken_triangular_couplings(beta, J, q)
    ea, eb, _ = triangular_bond_correlations(K1, K1, K2)
    return -J * (ea + eb), triangular_magnetization(K1, K1, K2)


def shaken_lattice_beta_c(J: float, q: float) -> float:
    """Critical beta of the lattice shaken chain (its doubling graph is hexagonal):
    tanh^2(beta J) + 2 tanh(beta J) tanh(beta q) = 1."""
    from scipy.optimize import brentq
    return float(brentq(lambda b: np.tanh(b * J) ** 2 + 2 * np.tanh(b * J) * np.tanh(b * q) - 1,
                        1e-6, 50.0))


def triangular_heat_bath(L: int, J: float, q: float, beta: float, sweeps: int, burn: int,
                         seed: int, start_plus: bool = False):
    """Single-spin heat bath on the anisotropic triangular Ising model that the
    lambda = 0 shaken measure equals (couplings K1 on (x, x_down) and (x, x_left),
    K2 on (x_down, x_left); see ``triangular_gibbs_lambda0``).  Sites are updated
    by colour class c = (i + 2 j) mod 3 (a proper colouring of that lattice when
    3 | L), so each class update is an exact Gibbs step.  Returns per-sweep
    samples of the square-lattice energy per site -(J/N) sum_x s_x (s_down + s_left)
    and of the magnetisation per site."""
    assert L % 3 == 0
    K, Q = beta * J, beta * q
    K1 = 0.25 * np.log(np.cosh(2 * K + Q) / np.cosh(2 * K - Q))
    K2 = 0.25 * np.log(np.cosh(2 * K + Q) * np.cosh(2 * K - Q) / np.cosh(Q) ** 2)
    g = np.random.default_rng(seed)
    s = np.ones((L, L)) if start_plus else np.where(g.random((L, L)) < 0.5, -1.0, 1.0)
    i, j = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    colour = (i + 2 * j) % 3
    masks = [colour == c for c in range(3)]
    E, M = [], []
    for sw in range(burn + sweeps):
        for c in range(3):
            # local field: K1 bonds to the four square neighbours, K2 bonds along (1,-1)
            f = K1 * (np.roll(s, 1, 0) + np.roll(s, -1, 0) + np.roll(s, 1, 1) + np.roll(s, -1, 1)) \
                + K2 * (np.roll(np.roll(s, 1, 0), -1, 1) + np.roll(np.roll(s, -1, 0), 1, 1))
            p = 1.0 / (1.0 + np.exp(-2.0 * f))
            new = np.where(g.random((L, L)) < p, 1.0, -1.0)
            s = np.where(masks[c], new, s)
        if sw >= burn:
            E.append(-J * np.mean(s * (np.roll(s, 1, 0) + np.roll(s, 1, 1))))
            M.append(np.mean(s))
    return np.array(E), np.array(M)


def batch_means_se(x: np.ndarray, nb: int = 20) -> float:
    """Standard error of the mean of a correlated series by batch means."""
    x = np.asarray(x)
    b = x[: len(x) // nb * nb].reshape(nb, -1).mean(axis=1)
    return float(b.std(ddof=1) / np.sqrt(nb))
