"""Pins of the plain-C oracle (oracle/shaken_oracle.c) to things fixed outside it.
CPU only.

* Philox-4x32-10 against an independent implementation (Triton's ``tl.philox``
  run by the Triton CPU interpreter) and the draw layouts against their
  definition assembled from that independent generator.
* Philox-4x32-10 against NVIDIA's cuRAND host generator (run on the CPU through
  its C API), under the key (seed low word, seed high word).
* The exponential against libm (<= 2 ulp) and exact values; the threshold
  T = floor(2^32 / (1 + e^{-2 beta h})) against a 60-digit evaluation (+-1) and
  its exact values at h = 0 and in saturation.
* The worked trajectory of the proof of Thm 3.3 (tests/golden), bit-exact.
* The oracle's stochastic half steps against the exact transition law
  mu_0 (P^{sh})^t (oracle/exact.py) by chi-square, on the lattice (both lane
  layouts, with and without a frozen set) and on a small graph (+-1 and real
  couplings).
* The first exit from the all-minus state: per-site flip probability
  1 / (1 + e^{2 beta (2J + q - lambda)}) (proof of Thm 3.3), binomial test.
* Observables against the independent numpy Hamiltonians of oracle/exact.py.
"""
import ctypes
import ctypes.util
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

from oracle import core, exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- Philox
def _triton_philox(seed, ctrs):
    pytest.importorskip("triton")
    req = json.dumps({"seed": int(seed), "ctrs": np.asarray(ctrs, dtype=np.int64).tolist()})
    script = os.path.join(os.path.dirname(__file__), "triton_philox_ref.py")
    res = subprocess.run([sys.executable, script], input=req, capture_output=True, text=True,
                         timeout=600)
    if res.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + res.stderr.strip().splitlines()[-1])
    return np.asarray(json.loads(res.stdout), dtype=np.int64).astype(np.uint32)


def test_philox_matches_independent_implementation():
    g = np.random.default_rng(1)
    ctrs = g.integers(0, 2**32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
    ctrs[0] = 0
    ctrs[1] = 0xFFFFFFFF
    for seed in (0, 12345, 0x5348414B, 2**32 + 7, 2**63 + 99):
        ref = _triton_philox(seed, ctrs)
        key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
        mine = np.array([core.philox(key, c) for c in ctrs])
        assert np.array_equal(mine, ref), seed


def _curand():
    names = [ctypes.util.find_library("curand"), "libcurand.so", "libcurand.so.10"]
    names += [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), d, "libcurand.so")
              for d in ("lib64", "lib")]
    for name in names:
        if not name:
            continue
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("libcurand not found")


def _curand_philox_host(lib, seed, offset, n):
    """n 32-bit outputs of cuRAND's host-side PHILOX4_32_10 generator (generator
    type 161 in curand.h) for `seed`, starting at output `offset`."""
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


def test_philox_matches_curand_host_generator():
    """A second implementation outside this project.  Its output block b (outputs
    4b .. 4b+3) is the Philox block of counter (p mod 2^32, p >> 32, s, 0) with
    s = b mod 2^16 and p = b >> 16 (65,536 subsequences in counter word 2, the
    position in words 0 and 1), so counter words 0, 1 and 2 and both key words are
    exercised; two consecutive blocks from each offset."""
    lib = _curand()
    for seed in (0, 1, 0x5348414B, 2**32 + 7, 0x123456789ABCDEF0, 2**64 - 1):
        key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
        for block in (0, 77, 65535, 65536 + 3, 2**31 + 3, 2**32 - 1, 2**48 + 5 * 65536 + 9):
            got = _curand_philox_host(lib, seed, 4 * block, 8).reshape(2, 4)
            for i in range(2):
                b = block + i
                p, sub = b >> 16, b & 0xFFFF
                ref = core.philox(key, [p & 0xFFFFFFFF, p >> 32, sub, 0])
                assert np.array_equal(got[i], ref), (seed, b)


def test_draw_layouts_match_definition():
    seed = 0x5348414B + 3
    ctrs = []
    a, b, t, half = 17, 5, 9, 1
    for c in range(8):
        ctrs.append([a, b, t, half + 2 * c])
    W = _triton_philox(seed, ctrs).reshape(-1)  # W_j = call j>>2, word j&3
    for k in range(32):
        u = 0
        for j in range(32):
            u |= ((int(W[j]) >> k) & 1) << (31 - j)
        assert core.draw_plane(seed, a, b, t, half, k) == u
        assert core.draw_direct(seed, a, b, t, half, k) == int(W[k])
        # graph lane words: vertex a, replica 32 b + k
        assert core.graph_draw(seed, a, 32 * b + k, t, half, core.DRAW_PLANE) == u
        assert core.graph_draw(seed, a, 32 * b + k, t, half, core.DRAW_DIRECT) == int(W[k])


def test_graph_fields_match_dense_form():
    # the per-vertex field sums (incidence lists, edge order) against the dense
    # oriented coupling matrix of oracle/exact.py: J^{oT} sigma (half 0) and
    # J^o sigma (half 1), plus q sigma + lambda (Sec. 2, fields below Eq. (ham21))
    g = np.random.default_rng(12)
    n, m = 40, 150
    u = g.integers(0, n, m).astype(np.int32)
    v = ((u + 1 + g.integers(0, n - 1, m)) % n).astype(np.int32)
    for integer_J in (True, False):
        J = np.where(g.random(m) < 0.5, -1.0, 1.0) if integer_J else g.standard_normal(m)
        lam = 0.3 * g.standard_normal(n)
        q = 0.7
        for rule in (0, 2):
            tail, head = core.orient(u, v, rule)
            Jo = exact.oriented_matrix(n, tail, head, J)
            s = np.where(g.random((5, n)) < 0.5, -1, 1).astype(np.int8)
            for half in (0, 1):
                h = core.graph_fields(s, tail, head, J, integer_J, lam, q, half)
                ref = exact.fields(s.astype(np.float64), Jo, lam, q, half)
                assert np.abs(h - ref).max() < 1e-12
                inc = core.Incidence(n, tail, head, J, integer_J, lam, q, half)
                for x in (0, 7, n - 1):
                    assert inc.field(s[2], x) == h[2, x]


def test_philox_output_is_uniform():
    key = np.array([7, 0], dtype=np.uint32)
    words = np.array([core.philox(key, [i, 0, 0, 0]) for i in range(4096)]).reshape(-1)
    # 8 equal bins of the top three bits
    counts = np.bincount(words >> 29, minlength=8)
    assert stats.chisquare(counts).pvalue > 1e-4
    bits = ((words[:, None] >> np.arange(32)) & 1).mean(axis=0)
    assert np.abs(bits - 0.5).max() < 5 * 0.5 / math.sqrt(words.size)


# --------------------------------------------------------------------------- exp and thresholds
def _ulp_diff(a, b):
    ia = np.frombuffer(np.float64(a).tobytes(), dtype=np.int64)[0]
    ib = np.frombuffer(np.float64(b).tobytes(), dtype=np.int64)[0]
    return abs(int(ia) - int(ib))


def test_exp_close_to_libm():
    g = np.random.default_rng(2)
    xs = np.concatenate([g.uniform(-63.9, 63.9, 20000), g.uniform(-1, 1, 5000),
                         np.arange(-63, 64, dtype=float) * math.log(2)])
    worst = max(_ulp_diff(core.exp(x), math.exp(x)) for x in xs)
    assert worst <= 2
    assert core.exp(0.0) == 1.0
    assert core.exp(-64.0) == 0.0 and math.isinf(core.exp(64.0))


def test_threshold_exact_points_and_saturation():
    for beta in (0.1, 0.4407, 1.0, 3.0):
        assert core.threshold(0.0, beta) == 2**31
    assert core.threshold(7.0, 3.0) == 2**32  # p rounds to 1
    assert core.threshold(-20.0, 3.0) == 0
    assert core.threshold(1.0, 0.0) == 2**31


def test_threshold_against_high_precision():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    g = np.random.default_rng(3)
    for _ in range(3000):
        h = float(g.uniform(-8, 8))
        beta = float(g.uniform(0.05, 3.0))
        y = beta * h  # the oracle rounds beta*h once, then works exactly up to 1 ulp of e
        ref = mpmath.floor(mpmath.mpf(2) ** 32 / (1 + mpmath.exp(-2 * mpmath.mpf(y))))
        T = core.threshold(h, beta)
        assert abs(T - int(ref)) <= 1, (h, beta)


def test_threshold_monotone_and_antisymmetric():
    hs = np.linspace(-6, 6, 2001)
    for beta in (0.3, 0.6, 2.0):
        T = np.array([core.threshold(h, beta) for h in hs], dtype=np.int64)
        assert np.all(np.diff(T) >= 0)
        Tm = np.array([core.threshold(-h, beta) for h in hs], dtype=np.int64)
        assert np.abs(T + Tm - 2**32).max() <= 2


def test_field_rounding_order():
    assert core.field(1.0, -2, 0.25, -1, 0.5) == (-2.0 + -0.25) + 0.5
    assert core.field(0.3, 2, 0.1, 1, 0.7) == (0.3 * 2 + 0.1) + 0.7


# --------------------------------------------------------------------------- worked example
def _golden_worked():
    spec = {}
    with open(os.path.join(GOLDEN, "worked_example_thm33.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split(":", 1)
            spec[k.strip()] = v.split()
    return spec


def _plus_set(s):
    return set(zip(*np.nonzero(s > 0)))


@pytest.mark.parametrize("L,i,j", [(8, 2, 3), (16, 0, 0), (32, 31, 5), (12, 7, 11)])
@pytest.mark.parametrize("mode", [core.MODE_SINGLE, core.MODE_MULTISPIN])
def test_worked_trajectory_thm33(L, i, j, mode):
    spec = _golden_worked()
    J, lam, q, beta = 1.0, 0.5, 0.25, 100.0  # 0 < q < lambda < J, every T in {0, 2^32}
    for s_ in (-1, 1):
        for n in (0, 1, 2):
            h = core.field(J, 2 * n - 2, q, s_, lam)
            assert core.threshold(h, beta) in (0, 2**32)
    s = -np.ones((1, L, L), dtype=np.int8)
    s[0, i, j] = 1

    def offs(key):
        return {((i + int(a)) % L, (j + int(b)) % L)
                for a, b in (p.split(",") for p in spec[key])}

    assert _plus_set(s[0]) == offs("initial")
    sp = core.lattice_half(s, J, q, lam, beta, seed=1, t=0, half=0, mode=mode)
    assert _plus_set(sp[0]) == offs("after_half_dl")
    s1 = core.lattice_half(sp, J, q, lam, beta, seed=1, t=0, half=1, mode=mode)
    assert _plus_set(s1[0]) == offs("after_full_step")
    assert spec["after_floor_L_over_2_full_steps"] == ["diagonal"]
    sf, _ = core.lattice_run(s, J, q, lam, beta, seed=1, t0=0, n_steps=L // 2, mode=mode)
    diag = {(a, b) for a in range(L) for b in range(L) if (a + b) % L == (i + j) % L}
    assert _plus_set(sf[0]) == diag
    # configurations in D are fixed points of the full step
    sf2, _ = core.lattice_run(sf, J, q, lam, beta, seed=1, t0=L // 2, n_steps=3, mode=mode)
    assert np.array_equal(sf2, sf)


def test_worked_trajectory_through_graph_path():
    L, i, j = 8, 2, 3
    u, v = exact.lattice_edges(L)  # oriented (x -> up), (x -> right)
    J = np.ones(u.size)
    s = -np.ones((32, L * L), dtype=np.int8)
    s[:, i * L + j] = 1
    sp = core.graph_half(s, u, v, J, True, 0.5, 0.25, 100.0, seed=3, t=0, half=0)
    got = {divmod(int(x), L) for x in np.nonzero(sp[0] > 0)[0]}
    assert got == {(i, j + 1), (i + 1, j)}
    sf, _ = core.graph_run(s, u, v, J, True, 0.5, 0.25, 100.0, seed=3, t0=0, n_steps=L // 2)
    got = {divmod(int(x), L) for x in np.nonzero(sf[5] > 0)[0]}
    assert got == {(a, b) for a in range(L) for b in range(L) if (a + b) % L == (i + j) % L}


def test_orientation_rule_min_to_max():
    u = np.array([5, 1, 7, 2], dtype=np.int32)
    v = np.array([3, 4, 0, 9], dtype=np.int32)
    t, h = core.orient(u, v, 0)
    assert list(t) == [3, 1, 0, 2] and list(h) == [5, 4, 7, 9]
    t, h = core.orient(u, v, 2)
    assert list(t) == list(u) and list(h) == list(v)


# --------------------------------------------------------------------------- chi-square vs exact law
def _chi2_pvalue(counts, probs, nrep):
    exp_ = probs * nrep
    big = exp_ >= 5
    obs = np.append(counts[big], counts[~big].sum())
    ex = np.append(exp_[big], exp_[~big].sum())
    if ex[-1] == 0:
        obs, ex = obs[:-1], ex[:-1]
    return stats.chisquare(obs, ex * obs.sum() / ex.sum()).pvalue


@pytest.mark.parametrize("mode", [core.MODE_SINGLE, core.MODE_MULTISPIN])
@pytest.mark.parametrize("frozen", [None, (0, 4)])
def test_lattice_chain_follows_exact_law(mode, frozen):
    L, R = 3, 6400
    J, q, lam, beta = 1.0, 0.7, 0.3, 0.6
    tails, heads = exact.lattice_edges(L)
    S = exact.states(L * L)
    Jo = exact.oriented_matrix(L * L, tails, heads, J)
    fz = None
    if frozen is not None:
        fz = np.zeros(L * L, dtype=np.uint8)
        fz[list(frozen)] = 1
    P = exact.shaken_matrix(S, Jo, lam, q, beta, frozen=None if fz is None else fz.astype(bool))
    s0 = np.array([1, -1, -1, 1, 1, -1, 1, -1, -1], dtype=np.int8)
    if fz is not None:
        s0[fz > 0] = 1
    mu0 = np.zeros(S.shape[0])
    mu0[exact.state_index(s0)] = 1.0
    s = np.broadcast_to(s0.reshape(1, L, L), (R, L, L)).copy()
    for t in (1, 3):
        st, _ = core.lattice_run(s, J, q, lam, beta, seed=0x5348414B + t, t0=11, n_steps=t,
                                 mode=mode, frozen=fz)
        idx = exact.state_index(st.reshape(R, -1))
        counts = np.bincount(idx, minlength=S.shape[0]).astype(float)
        assert _chi2_pvalue(counts, exact.evolve(mu0, P, t), R) > 1e-4


@pytest.mark.parametrize("integer_J,draw", [(True, core.DRAW_DIRECT), (False, core.DRAW_DIRECT),
                                            (True, core.DRAW_PLANE)])
def test_graph_chain_follows_exact_law(integer_J, draw):
    n, R = 6, 6400
    u = np.array([0, 1, 2, 3, 4, 5, 0, 2], dtype=np.int32)
    v = np.array([1, 2, 3, 4, 5, 0, 3, 5], dtype=np.int32)
    g = np.random.default_rng(5)
    J = np.where(g.random(8) < 0.5, -1.0, 1.0) if integer_J else g.standard_normal(8)
    lam = 0.3 * g.standard_normal(n)
    q, beta = 0.8, 0.7
    tail, head = core.orient(u, v, 0)
    S = exact.states(n)
    Jo = exact.oriented_matrix(n, tail, head, J)
    P = exact.shaken_matrix(S, Jo, lam, q, beta)
    s0 = np.array([1, 1, -1, -1, 1, -1], dtype=np.int8)
    mu0 = np.zeros(S.shape[0])
    mu0[exact.state_index(s0)] = 1.0
    s = np.broadcast_to(s0, (R, n)).copy()
    for t in (1, 2):
        st, _ = core.graph_run(s, tail, head, J, integer_J, lam, q, beta, seed=77 + t, t0=3,
                               n_steps=t, draw=draw)
        counts = np.bincount(exact.state_index(st), minlength=S.shape[0]).astype(float)
        assert _chi2_pvalue(counts, exact.evolve(mu0, P, t), R) > 1e-4


def test_random_init_is_fair():
    s = core.lattice_init(64, 4, seed=9, mode=core.MODE_SINGLE, kind=0)
    k = int((s > 0).sum())
    assert abs(k - s.size / 2) < 5 * math.sqrt(s.size) / 2
    s = core.graph_init(1000, 64, seed=9, kind=0)
    k = int((s > 0).sum())
    assert abs(k - s.size / 2) < 5 * math.sqrt(s.size) / 2


def test_first_exit_probability_from_minus():
    # proof of Thm 3.3: from -1 a site flips in the dl half step with probability
    # 1 / (1 + e^{2 beta (2J + q - lambda)})
    J, q, lam, beta = 1.0, 0.1, 0.15, 0.5
    L, R = 32, 64
    s = -np.ones((R, L, L), dtype=np.int8)
    sp = core.lattice_half(s, J, q, lam, beta, seed=21, t=0, half=0)
    p = 1.0 / (1.0 + math.exp(2 * beta * (2 * J + q - lam)))
    k = int((sp > 0).sum())
    N = sp.size
    assert stats.binomtest(k, N, p).pvalue > 1e-4


def exit_probability_per_step(J, q, lam, beta, N):
    """P(sigma_{t+1} != -1 | sigma_t = -1) on an N-site torus, to first order in the
    single-site flip probability p0 (proof of Thm 3.3).  Half dl from -1: every site
    has h0 = -2J - q + lambda.  If sigma' = -1, half ur gives h0 again.  If sigma' has
    one + at x, half ur gives x the field h1 = -2J + q + lambda, the two sites below
    and left of x (whose up / right neighbour is x) h2 = lambda - q, the rest h0.
    Terms with two or more flips, O((N p0)^2), are dropped."""
    def p(h):
        return 1.0 / (1.0 + math.exp(-2.0 * beta * h))
    p0, p1, p2 = p(-2 * J - q + lam), p(-2 * J + q + lam), p(lam - q)
    stay = (1 - p0) ** (2 * N)
    stay += N * p0 * (1 - p0) ** (N - 1) * (1 - p1) * (1 - p2) ** 2 * (1 - p0) ** (N - 3)
    return 1.0 - stay


def exit_rate_mle(first, T):
    """Censored geometric MLE of the per-step exit probability: exits / exposure, with
    `first` the step (1-based) of each replica's first exit, 0 if none by step T."""
    first = np.asarray(first)
    exits = int((first > 0).sum())
    exposure = float(np.where(first > 0, first, T).sum())
    return exits / exposure, exits


def test_exit_time_from_minus_matches_first_order_law():
    """Full steps from -1 (J = 1, q = 0.1, lambda = 0.15: the regime 0 < q < lambda < J
    of Thm 3.1) until the first full-step configuration other than -1: geometric with
    the per-step probability of exit_probability_per_step."""
    J, q, lam, beta = 1.0, 0.1, 0.15, 2.5
    L, R, T = 16, 128, 150
    s = core.lattice_init(L, R, 0x5348414B + 5, core.MODE_SINGLE, kind=2)
    first = np.zeros(R, dtype=np.int64)
    for t in range(1, T + 1):
        s, _ = core.lattice_run(s, J, q, lam, beta, 0x5348414B + 5, t - 1, 1, core.MODE_SINGLE)
        out = (s.reshape(R, -1) > 0).any(axis=1)
        first[(first == 0) & out] = t
    P = exit_probability_per_step(J, q, lam, beta, L * L)
    Phat, exits = exit_rate_mle(first, T)
    assert abs(Phat - P) < 4 * Phat / math.sqrt(exits), (Phat, P, exits)


# --------------------------------------------------------------------------- observables
def test_lattice_sums_match_numpy_hamiltonians():
    L = 5
    J, q, lam = 0.9, 0.4, 0.2
    tails, heads = exact.lattice_edges(L)
    g = np.random.default_rng(8)
    for _ in range(20):
        s = np.where(g.random((L, L)) < 0.5, -1, 1).astype(np.int8)
        sp = np.where(g.random((L, L)) < 0.5, -1, 1).astype(np.int8)
        obs = core.lattice_observables(s[None], sp[None], J, q, lam)[0]
        H = exact.hamiltonian(s.reshape(1, -1).astype(np.int64), tails, heads, J, lam)[0]
        Hp = exact.pair_hamiltonian(s.reshape(1, -1).astype(np.int64),
                                    sp.reshape(1, -1).astype(np.int64), tails, heads, J, lam, q)[0]
        assert abs(obs["H"] - H) < 1e-12 and abs(obs["pair"] - Hp) < 1e-12
        ss = s.reshape(-1).astype(np.int64)
        assert obs["cut"] == int((ss[tails] != ss[heads]).sum())
        same = core.lattice_observables(s[None], s[None], J, q, lam)[0]
        assert abs(same["pair"] - (same["H"] - q * L * L)) < 1e-12


def test_graph_sums_match_numpy_hamiltonians():
    n = 7
    u = np.array([0, 1, 2, 3, 4, 5, 6, 0, 2], dtype=np.int32)
    v = np.array([1, 2, 3, 4, 5, 6, 0, 3, 6], dtype=np.int32)
    g = np.random.default_rng(9)
    J = g.standard_normal(u.size)
    lam = g.standard_normal(n)
    q = 0.55
    tail, head = core.orient(u, v, 0)
    for _ in range(10):
        s = np.where(g.random((1, n)) < 0.5, -1, 1).astype(np.int8)
        sp = np.where(g.random((1, n)) < 0.5, -1, 1).astype(np.int8)
        o = core.graph_observables(s, sp, tail, head, J, lam, q)[0]
        H = exact.hamiltonian(s.astype(np.int64), tail, head, J, lam)[0]
        Hp = exact.pair_hamiltonian(s.astype(np.int64), sp.astype(np.int64), tail, head, J, lam,
                                    q)[0]
        assert abs(o["H"] - H) < 1e-12 and abs(o["pair"] - Hp) < 1e-12
