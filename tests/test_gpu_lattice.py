"""Lattice parity: the CUDA kernels (INT8, PACKED, MULTISPIN encodings) against
the CPU oracle, bit for bit, on the same seeded inputs (Sec. 3 of
arXiv:1904.06257: P^dl then P^ur on the L x L torus, frozen set B)."""
import numpy as np
import pytest

from oracle import core
from paper_1904_06257_gb300 import workloads as W
from tests.gpu_util import lattice_problem, lib, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    require_cuda()
    return lib()


def mode_of(S, enc):
    return core.MODE_MULTISPIN if enc == S.MULTISPIN else core.MODE_SINGLE


CASES = [
    # enc, L, R, J, q, lam, frozen
    ("INT8", 64, 1, 1.0, 1.0, 0.0, False),
    ("INT8", 96, 3, 1.0, 0.5, 0.01, False),     # 288 lane words: 2 tiles, ragged tail
    ("INT8", 160, 2, 0.7, 2.0, -0.3, True),
    ("PACKED", 96, 3, 1.0, 0.5, 0.01, False),
    ("PACKED", 64, 2, -1.0, 1.0, 0.2, True),
    ("MULTISPIN", 32, 64, 1.0, 1.0, 0.0, False),
    ("MULTISPIN", 96, 32, 1.0, 0.5, 0.01, True),  # 9216 sites: 36 tiles
    ("MULTISPIN", 160, 64, 0.8, 0.7, 0.05, True),  # 25600 sites x 2 groups, frozen frame
]


@pytest.mark.parametrize("enc,L,R,J,q,lam,frozen", CASES)
def test_trajectory_bit_exact(S, enc, L, R, J, q, lam, frozen):
    e = getattr(S, enc)
    beta = W.beta_grid(R, 0.3, 0.6, 7)
    fz = W.frozen_frame(L) if frozen else None
    seed = 0x5348414B + L + R
    ctx = S.shaken_init(lattice_problem(S, e, L, R, beta, J, q, lam, fz), seed)
    try:
        s0 = S.shaken_get_spins(ctx, R, L * L).reshape(R, L, L)
        o0 = core.lattice_init(L, R, seed, mode_of(S, e), 0, fz)
        assert np.array_equal(s0, o0), "initial configuration"
        steps = 6
        S.shaken_step(ctx, steps)
        s1 = S.shaken_get_spins(ctx, R, L * L).reshape(R, L, L)
        o1, osp = core.lattice_run(o0, J, q, lam, beta, seed, 0, steps, mode_of(S, e), fz)
        assert np.array_equal(s1, o1)
        assert S.shaken_get_step(ctx) == steps
        # observables (sigma, sigma') against the oracle's integer sums
        obs = S.shaken_observables(ctx, R)
        ref = core.lattice_observables(o1, osp, J, q, lam)
        for r in range(R):
            assert abs(obs["magnetization"][r] - ref[r]["m"]) < 1e-12
            assert abs(obs["energy"][r] - ref[r]["H"]) < 1e-9
            assert abs(obs["pair_energy"][r] - ref[r]["pair"]) < 1e-9
            assert obs["cut_edges"][r] == ref[r]["cut"]
    finally:
        S.shaken_free(ctx)


@pytest.mark.parametrize("L", [32, 64, 128])
def test_int8_and_packed_identical(S, L):
    R = 2
    beta = [0.44, 0.5]
    out = []
    for e in (S.INT8, S.PACKED):
        ctx = S.shaken_init(lattice_problem(S, e, L, R, beta, 1.0, 1.0, 0.0), 99)
        S.shaken_step(ctx, 40)
        out.append(S.shaken_get_spins(ctx, R, L * L))
        S.shaken_free(ctx)
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("enc", ["INT8", "PACKED", "MULTISPIN"])
def test_worked_trajectory_thm33_on_gpu(S, enc):
    # proof of Thm 3.3: single + spin grows into its diagonal in [L/2] steps
    e = getattr(S, enc)
    L, R = 64, (32 if enc == "MULTISPIN" else 1)
    i, j = 10, 17
    init = -np.ones((R, L, L), dtype=np.int8)
    init[:, i, j] = 1
    ctx = S.shaken_init(lattice_problem(S, e, L, R, 100.0, 1.0, 0.25, 0.5, init=S.INIT_GIVEN,
                                        init_spins=init.reshape(R, -1)), 5)
    S.shaken_step(ctx, L // 2)
    s = S.shaken_get_spins(ctx, R, L * L).reshape(R, L, L)
    a, b = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    diag = np.where((a + b) % L == (i + j) % L, 1, -1)
    assert all(np.array_equal(s[r], diag) for r in range(R))
    S.shaken_free(ctx)


@pytest.mark.parametrize("enc", ["INT8", "MULTISPIN"])
def test_anneal_bit_exact_and_best(S, enc):
    e = getattr(S, enc)
    L, R = 64, (32 if enc == "MULTISPIN" else 2)
    J, q, lam = 1.0, 1.0, 0.05
    sched = W.linear_schedule(0.1, 1.5, 12)
    seed = 4242
    ctx = S.shaken_init(lattice_problem(S, e, L, R, 0.4, J, q, lam), seed)
    S.shaken_step(ctx, 3)
    S.shaken_anneal(ctx, sched)
    s = S.shaken_get_spins(ctx, R, L * L).reshape(R, L, L)
    o = core.lattice_init(L, R, seed, mode_of(S, e), 0)
    o, _ = core.lattice_run(o, J, q, lam, 0.4, seed, 0, 3, mode_of(S, e))
    best = np.full(R, np.inf)
    cur = o.copy()
    for k, b in enumerate(sched):
        for r in range(R):
            H = core.lattice_observables(cur[r:r + 1], cur[r:r + 1], J, q, lam)[0]["H"]
            best[r] = min(best[r], H)
        cur, _ = core.lattice_run(cur, J, q, lam, b, seed, 3 + k, 1, mode_of(S, e))
    assert np.array_equal(s, cur)
    obs = S.shaken_observables(ctx, R)
    for r in range(R):
        Hf = core.lattice_observables(cur[r:r + 1], cur[r:r + 1], J, q, lam)[0]["H"]
        assert abs(obs["best_energy"][r] - min(best[r], Hf)) < 1e-9
    S.shaken_free(ctx)


def test_step_record_series(S):
    L, R = 64, 2
    J, q, lam = 1.0, 1.0, 0.01
    seed = 77
    ctx = S.shaken_init(lattice_problem(S, S.INT8, L, R, [0.4, 0.45], J, q, lam), seed)
    mag, en = S.shaken_step_record(ctx, 8, R)
    cur = core.lattice_init(L, R, seed, core.MODE_SINGLE, 0)
    for k in range(8):
        for r in range(R):
            ob = core.lattice_observables(cur[r:r + 1], cur[r:r + 1], J, q, lam)[0]
            assert abs(mag[k, r] - ob["m"]) < 1e-12
            assert abs(en[k, r] - ob["H"]) < 1e-9
        cur, _ = core.lattice_run(cur, J, q, lam, [0.4, 0.45], seed, k, 1, core.MODE_SINGLE)
    S.shaken_free(ctx)


@pytest.mark.parametrize("enc", ["INT8", "PACKED", "MULTISPIN"])
def test_full_size_sampled_sites(S, enc):
    """L = 4096 (the plain single-lattice size; multispin: 32 replicas of 1024^2),
    one half step in the bench's launch configuration, checked at sampled sites
    against the oracle's single-site update."""
    e = getattr(S, enc)
    L, R = (4096, 1) if enc != "MULTISPIN" else (1024, 32)
    J, q, lam, beta = 1.0, 1.0, 0.01, 0.4407
    seed = 0x5348414B
    ctx = S.shaken_init(lattice_problem(S, e, L, R, beta, J, q, lam), seed)
    s0 = S.shaken_get_spins(ctx, R, L * L).reshape(R, L, L)
    S.shaken_step(ctx, 1)
    s1 = S.shaken_get_spins(ctx, R, L * L).reshape(R, L, L)
    g = np.random.default_rng(3)
    mode = mode_of(S, e)
    for _ in range(300):
        r = int(g.integers(R))
        i, j = int(g.integers(L)), int(g.integers(L))
        # neighbourhood of the half-step-1 update needs sigma' at (i,j),(i+1,j),(i,j+1)
        sp = {}
        for (a, b) in ((i, j), ((i + 1) % L, j), (i, (j + 1) % L)):
            sp[(a, b)] = core.lattice_site(s0[r], a, b, J, q, lam, beta, seed, 0, 0, mode, r)
        # rebuild a local copy of sigma' around (i, j) and evaluate the second half step
        loc = s0[r]
        saved = {k: loc[k] for k in sp}
        for (a, b), v in sp.items():
            loc[a, b] = v
        tau = core.lattice_site(loc, i, j, J, q, lam, beta, seed, 0, 1, mode, r)
        for k, v in saved.items():
            loc[k] = v
        assert s1[r, i, j] == tau
    S.shaken_free(ctx)


def test_frozen_sites_stay_plus(S):
    L = 64
    fz = W.frozen_frame(L)
    ctx = S.shaken_init(lattice_problem(S, S.PACKED, L, 1, 0.3, 1.0, 1.0, -0.5, fz), 3)
    S.shaken_step(ctx, 20)
    s = S.shaken_get_spins(ctx, 1, L * L)[0]
    assert np.all(s[fz > 0] == 1)
    S.shaken_free(ctx)


@pytest.mark.parametrize("enc", ["INT8", "PACKED", "MULTISPIN"])
def test_tiled_and_resident_paths_agree_with_oracle(S, enc):
    """Small lattices run chunks of >= 4 steps in one resident launch; chunks of
    fewer steps use the per-half-step tiled kernels.  Both must follow the oracle."""
    e = getattr(S, enc)
    L, R = (64, 32) if enc == "MULTISPIN" else (96, 2)
    beta = W.beta_grid(R, 0.35, 0.5, 5)
    J, q, lam, seed = 1.0, 0.8, 0.02, 99
    ctx = S.shaken_init(lattice_problem(S, e, L, R, beta, J, q, lam), seed)
    mode = mode_of(S, e)
    o = core.lattice_init(L, R, seed, mode, 0)
    t = 0
    for n in (2, 5, 3, 1, 6):  # tiled, resident, tiled, tiled, resident
        S.shaken_step(ctx, n)
        o, _ = core.lattice_run(o, J, q, lam, beta, seed, t, n, mode)
        t += n
        assert np.array_equal(S.shaken_get_spins(ctx, R, L * L).reshape(R, L, L), o), n
    S.shaken_free(ctx)


@pytest.mark.parametrize("enc,L,frozen,order", [("INT8", 512, False, 0), ("PACKED", 512, True, 0),
                                               ("PACKED", 416, False, 1), ("INT8", 800, True, 1)])
def test_banded_path_agrees_with_oracle(S, enc, L, frozen, order):
    """Single lattices above the resident size run chunks of >= 8 steps in one
    cooperative launch holding the lattice in shared memory as row bands (halo rows
    exchanged between blocks through a grid barrier); chunks of fewer steps use the
    tiled kernels.  Both must follow the oracle: rows split unevenly (416, 800 are not
    multiples of the block count), a frozen frame, the reversed order P^{sh'}."""
    e = getattr(S, enc)
    J, q, lam, beta, seed = 1.0, 0.9, 0.03, 0.42, 4242 + L
    fz = W.frozen_frame(L) if frozen else None
    ctx = S.shaken_init(lattice_problem(S, e, L, 1, beta, J, q, lam, fz), seed)
    if order:
        S.shaken_set_order(ctx, 1)
    mode = mode_of(S, e)
    o = core.lattice_init(L, 1, seed, mode, 0, fz)
    sp = None
    t = 0
    for n in (9, 2, 8):  # banded, tiled, banded
        l0 = S.shaken_launch_count(ctx)
        S.shaken_step(ctx, n)
        if n >= 8:
            assert S.shaken_launch_count(ctx) - l0 == 1  # one banded launch
        if order:
            # reversed order: half ur then dl, draws keyed by update type
            for k in range(n):
                o1 = core.lattice_half(o, J, q, lam, beta, seed, t + k, 1, mode, fz)
                o = core.lattice_half(o1, J, q, lam, beta, seed, t + k, 0, mode, fz)
                sp = o1
        else:
            o, sp = core.lattice_run(o, J, q, lam, beta, seed, t, n, mode, fz)
        t += n
        got = S.shaken_get_spins(ctx, 1, L * L).reshape(1, L, L)
        assert np.array_equal(got, o), (n, int((got != o).sum()))
    obs = S.shaken_observables(ctx, 1)
    ref = core.lattice_observables(o, sp, J, q, lam)[0]
    assert abs(obs["magnetization"][0] - ref["m"]) < 1e-12
    assert abs(obs["pair_energy"][0] - ref["pair"]) < 1e-9
    S.shaken_free(ctx)


def test_banded_barrier_timeout_leaves_state(S):
    """Failure path of a banded run without a GPU fault: the diagnostic presets the
    grid barrier so that it never completes; every block's bounded wait runs out
    (about a second), the call returns E_TIMEOUT, sigma and the step counter are
    those before the call, and the context keeps stepping exactly as the oracle."""
    L, J, q, lam, beta, seed = 512, 1.0, 1.0, 0.0, 0.44, 606
    ctx = S.shaken_init(lattice_problem(S, S.PACKED, L, 1, beta, J, q, lam), seed)
    s0 = S.shaken_get_spins(ctx, 1, L * L)
    S.shaken_debug_band_stall(ctx)
    with pytest.raises(S.ShakenError) as err:
        S.shaken_step(ctx, 8)
    assert err.value.status == -4  # SHAKEN_E_TIMEOUT
    assert np.array_equal(S.shaken_get_spins(ctx, 1, L * L), s0)
    assert S.shaken_get_step(ctx) == 0
    S.shaken_step(ctx, 8)
    o = core.lattice_init(L, 1, seed, core.MODE_SINGLE, 0)
    o, _ = core.lattice_run(o, J, q, lam, beta, seed, 0, 8, core.MODE_SINGLE)
    assert np.array_equal(S.shaken_get_spins(ctx, 1, L * L).reshape(1, L, L), o)
    S.shaken_free(ctx)


def test_banded_timeout_at_last_barrier_is_all_or_nothing(S):
    """A block that gives up its wait at the last barrier while the other blocks are
    arriving or already through: the chunk's outcome is settled by one atomic
    decision, so the call either succeeds with the whole chunk applied (equal to the
    oracle's trajectory) or returns E_TIMEOUT with sigma, sigma' and the step counter
    exactly as before -- never a partly written chunk.  No wait is unbounded: the
    hurried block's deadline is zero, everyone else's one second."""
    L, J, q, lam, beta, seed = 512, 1.0, 1.0, 0.0, 0.44, 607
    ctx = S.shaken_init(lattice_problem(S, S.PACKED, L, 1, beta, J, q, lam), seed)
    o = core.lattice_init(L, 1, seed, core.MODE_SINGLE, 0)
    t = 0
    outcomes = set()
    for block in (0, 1, 5, 40, 100, 303, 0, 1):
        before = S.shaken_get_spins(ctx, 1, L * L)
        before_p = S.shaken_get_spins_prime(ctx, 1, L * L)
        S.shaken_debug_band_hurry(ctx, block)
        try:
            S.shaken_step(ctx, 8)
            outcomes.add("ok")
            o, op = core.lattice_run(o, J, q, lam, beta, seed, t, 8, core.MODE_SINGLE)
            t += 8
            assert np.array_equal(S.shaken_get_spins(ctx, 1, L * L).reshape(1, L, L), o)
            assert np.array_equal(S.shaken_get_spins_prime(ctx, 1, L * L).reshape(1, L, L), op)
        except S.ShakenError as err:
            assert err.status == -4  # SHAKEN_E_TIMEOUT
            outcomes.add("timeout")
            assert np.array_equal(S.shaken_get_spins(ctx, 1, L * L), before)
            assert np.array_equal(S.shaken_get_spins_prime(ctx, 1, L * L), before_p)
        assert S.shaken_get_step(ctx) == t
    S.shaken_free(ctx)
    assert outcomes  # at least one chunk ran; which outcomes occur depends on timing


@pytest.mark.parametrize("enc,L", [("INT8", 4096), ("PACKED", 8192)])
def test_banded_path_equals_tiled_path_at_full_size(S, enc, L):
    """At the plain-lattice size (4096^2, the bench's configuration) and at 8192^2
    (one band block per SM), 8 steps in one banded launch equal 8 single steps of the
    per-half-step tiled kernels, which the oracle pins at smaller sizes."""
    e = getattr(S, enc)
    J, q, lam, beta, seed = 1.0, 1.0, 0.0, 0.4407, 0x5348414B + L
    a = S.shaken_init(lattice_problem(S, e, L, 1, beta, J, q, lam), seed)
    b = S.shaken_init(lattice_problem(S, e, L, 1, beta, J, q, lam), seed)
    l0 = S.shaken_launch_count(a)
    S.shaken_step(a, 8)
    assert S.shaken_launch_count(a) - l0 == 1  # the banded path ran
    for _ in range(8):
        S.shaken_step(b, 1)
    assert np.array_equal(S.shaken_get_spins(a, 1, L * L), S.shaken_get_spins(b, 1, L * L))
    S.shaken_free(a)
    S.shaken_free(b)
