"""Seeded synthetic inputs for the shaken-dynamics workloads.

This module generates problem data only -- graphs, couplings, fields, inverse
temperatures, lattice sizes and serving streams -- and holds none of the
method's arithmetic (no fields, thresholds, draws or updates).  Both the CUDA
path (tests, bench) and the CPU oracle consume what it returns.

Workloads (sizes and distributions of the shaken-dynamics study, Sec. 3 and
Sec. 6 of arXiv:1904.06257, plus synthetic stand-ins for the Edwards-Anderson
instances the paper does not publish):

* square lattices L x L (periodic or with a frozen set), J = 1;
* batched multispin groups: L uniform over {32, 64, 128, 256, 512}, a beta grid
  of 64 values in [0.3, 0.6];
* random 3-regular graphs (configuration model with rejection) and
  Erdos-Renyi graphs of mean degree d (G(n, p), p = d / (n - 1));
* couplings J = +-1 i.i.d. or N(0, 1); fields lambda_x ~ N(0, sd);
* a Poisson stream of annealing jobs for the serving loop.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 0x5348414B  # "SHAK"


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def beta_grid(replicas: int, lo: float = 0.3, hi: float = 0.6, count: int = 64) -> np.ndarray:
    """beta_r = lo + (hi - lo) * (r mod count) / (count - 1)."""
    r = np.arange(replicas)
    return lo + (hi - lo) * (r % count) / (count - 1)


def multispin_group_sizes(groups: int, seed: int, choices=(32, 64, 128, 256, 512)) -> np.ndarray:
    """Side length of each 32-replica multispin group, uniform over ``choices``."""
    return rng(seed).choice(np.asarray(choices), size=groups)


def frozen_frame(L: int) -> np.ndarray:
    """Default frozen set: row 0 and column 0 of the L x L torus (uint8 mask)."""
    f = np.zeros((L, L), dtype=np.uint8)
    f[0, :] = 1
    f[:, 0] = 1
    return f.reshape(-1)


def _unique_sorted(keys: np.ndarray) -> np.ndarray:
    """Sorted distinct values (sort + neighbour comparison)."""
    k = np.sort(keys, kind="stable")
    if k.size == 0:
        return k
    keep = np.empty(k.size, dtype=bool)
    keep[0] = True
    np.not_equal(k[1:], k[:-1], out=keep[1:])
    return k[keep]


def random_regular3(n: int, seed: int, max_tries: int = 1000):
    """Random simple 3-regular graph on n (even) vertices: configuration model,
    rejecting pairings with loops or multi-edges."""
    if n % 2:
        raise ValueError("3-regular graph needs an even n")
    g = rng(seed)
    stubs = np.repeat(np.arange(n, dtype=np.int64), 3)
    for _ in range(max_tries):
        perm = g.permutation(stubs)
        u, v = perm[0::2], perm[1::2]
        if np.any(u == v):
            continue
        a, b = np.minimum(u, v), np.maximum(u, v)
        key = a * n + b
        if _unique_sorted(key).size != key.size:
            continue
        return a.astype(np.int32), b.astype(np.int32)
    # large n: repair by re-pairing only the bad stubs (rare) -- keeps it simple and exact
    raise RuntimeError("configuration model did not produce a simple graph")


def erdos_renyi(n: int, mean_degree: float, seed: int):
    """G(n, p) with p = mean_degree / (n - 1): the edge count is Binomial(n(n-1)/2, p)
    and the edges are a uniform sample of distinct pairs."""
    g = rng(seed)
    pairs = n * (n - 1) // 2
    p = mean_degree / (n - 1)
    m = int(g.binomial(pairs, p))
    keys = np.empty(0, dtype=np.int64)
    while keys.size < m:
        need = m - keys.size
        u = g.integers(0, n, size=int(need * 1.1) + 16, dtype=np.int64)
        v = g.integers(0, n, size=u.size, dtype=np.int64)
        ok = u != v
        a, b = np.minimum(u[ok], v[ok]), np.maximum(u[ok], v[ok])
        keys = _unique_sorted(np.concatenate([keys, a * n + b]))
    keys = g.permutation(keys)[:m]
    keys.sort()
    return (keys // n).astype(np.int32), (keys % n).astype(np.int32)


def power_law(n: int, mean_degree: float, exponent: float, seed: int):
    """Chung-Lu graph with a power-law degree sequence: vertex i has weight
    w_i ~ (i + 1)^(-1/(exponent - 1)), scaled to the mean degree; m = n mean_degree / 2
    edges are drawn with both ends chosen proportionally to the weights, and
    self-loops and repeated pairs are dropped.  Vertices of small index are hubs."""
    g = rng(seed)
    w = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (exponent - 1.0))
    p = w / w.sum()
    m = int(n * mean_degree / 2)
    u = g.choice(n, size=m, p=p).astype(np.int64)
    v = g.choice(n, size=m, p=p).astype(np.int64)
    ok = u != v
    a, b = np.minimum(u[ok], v[ok]), np.maximum(u[ok], v[ok])
    keys = _unique_sorted(a * n + b)
    return (keys // n).astype(np.int32), (keys % n).astype(np.int32)


def couplings_pm1(m: int, seed: int) -> np.ndarray:
    """J_e = +-1 with probability 1/2 each (float32)."""
    return np.where(rng(seed).random(m) < 0.5, -1.0, 1.0).astype(np.float32)


def couplings_normal(m: int, seed: int) -> np.ndarray:
    """J_e ~ N(0, 1) (float32)."""
    return rng(seed).standard_normal(m).astype(np.float32)


def fields_normal(n: int, sd: float, seed: int) -> np.ndarray:
    """lambda_x ~ N(0, sd^2) (float32)."""
    return (sd * rng(seed).standard_normal(n)).astype(np.float32)


def linear_schedule(lo: float, hi: float, steps: int) -> np.ndarray:
    """beta_t = lo + (hi - lo) t / (steps - 1), t = 0..steps-1."""
    if steps == 1:
        return np.array([hi], dtype=np.float64)
    return lo + (hi - lo) * np.arange(steps, dtype=np.float64) / (steps - 1)


def lattice_as_graph(L: int):
    """Edges of the L x L torus oriented by the lattice rule (x -> x_up, x -> x_right),
    x = (i, j) -> i*L + j, up = row i+1, right = column j+1."""
    i, j = np.divmod(np.arange(L * L), L)
    x = i * L + j
    up = ((i + 1) % L) * L + j
    rt = i * L + (j + 1) % L
    u = np.concatenate([x, x]).astype(np.int32)
    v = np.concatenate([up, rt]).astype(np.int32)
    return u, v


def triangular_lattice_as_graph(L: int):
    """Edges of the L x L triangular lattice (square lattice plus the (1,-1)
    diagonal, periodic), each oriented from x to its three "right" neighbours
    (i, j+1), (i+1, j), (i+1, j-1); the "left" neighbours are then the
    in-neighbours.  x = (i, j) -> i*L + j."""
    i, j = np.divmod(np.arange(L * L), L)
    x = i * L + j
    nb = [i * L + (j + 1) % L, ((i + 1) % L) * L + j, ((i + 1) % L) * L + (j - 1) % L]
    u = np.concatenate([x, x, x]).astype(np.int32)
    v = np.concatenate(nb).astype(np.int32)
    return u, v


def split_both_ways(u, v, J, frac=0.5):
    """Generalised decomposition J = J^o + J^oT: every edge {u, v} becomes the two
    oriented edges (u -> v) with weight frac J and (v -> u) with (1 - frac) J
    (frac = 1/2 is the symmetric PCA)."""
    uu = np.concatenate([u, v]).astype(np.int32)
    vv = np.concatenate([v, u]).astype(np.int32)
    JJ = np.concatenate([frac * np.asarray(J), (1 - frac) * np.asarray(J)]).astype(np.float32)
    return uu, vv, JJ


def serving_stream(rate_per_s: float, horizon_s: float, seed: int, n_lo=1_000, n_hi=1_000_000,
                   deg_lo=3.0, deg_hi=16.0, rep_lo=32, rep_hi=1024, steps_lo=1000,
                   steps_hi=20000, max_jobs=None):
    """Poisson arrivals of annealing jobs: n log-uniform in [n_lo, n_hi], mean degree
    uniform in [deg_lo, deg_hi], replicas log-uniform over multiples of 32 in
    [rep_lo, rep_hi], steps uniform in [steps_lo, steps_hi]."""
    g = rng(seed)
    t, jobs = 0.0, []
    while True:
        t += g.exponential(1.0 / rate_per_s)
        if t > horizon_s or (max_jobs is not None and len(jobs) >= max_jobs):
            break
        n = int(round(np.exp(g.uniform(np.log(n_lo), np.log(n_hi)))))
        n += n % 2
        deg = float(g.uniform(deg_lo, deg_hi))
        reps = int(np.exp(g.uniform(np.log(rep_lo), np.log(rep_hi))))
        reps = max(rep_lo, min(rep_hi, 32 * int(round(reps / 32))))
        steps = int(g.integers(steps_lo, steps_hi + 1))
        jobs.append(dict(arrival=t, n=n, mean_degree=deg, replicas=reps, steps=steps,
                         seed=BASE_SEED + len(jobs)))
    return jobs
