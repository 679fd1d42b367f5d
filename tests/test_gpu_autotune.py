"""Launch-shape autotuner and the bench's batched workload on the GPU.

The tuner times the lattice half-step kernel with 1 and 4 lane words per thread
by trial launches of the first half step; those launches must leave no trace in
any trajectory, and every shape must give the oracle's decisions."""
import numpy as np
import pytest

from oracle import core
from paper_1904_06257_gb300 import workloads as W
from tests.gpu_util import lattice_problem, lib, require_cuda

pytestmark = pytest.mark.gpu

# the batched multispin workload: 128 groups of 32 replicas, L uniform in {32..512},
# beta grid of 64 in [0.3, 0.6], J = q = 1, lambda = 0
GROUPS, L_CHOICES = 128, (32, 64, 128, 256, 512)


@pytest.fixture(scope="module")
def S():
    require_cuda()
    return lib()


def batch_of(S, Ls, betas, seeds, autotune):
    b = S.shaken_batch_create()
    S.shaken_batch_set_autotune(b, autotune)
    ctxs = []
    for g, L in enumerate(Ls):
        c = S.shaken_init(lattice_problem(S, S.MULTISPIN, int(L), 32, betas[32 * g:32 * g + 32]),
                          seeds[g])
        S.shaken_batch_add(b, c)
        ctxs.append(c)
    return b, ctxs


def free_batch(S, b, ctxs):
    for c in ctxs:
        S.shaken_batch_remove(b, c)
        S.shaken_free(c)
    S.shaken_batch_free(b)


def test_trials_leave_no_trace_and_results_are_cached(S):
    """Two 512 x 512 groups (524,288 lane words: one wave of 1024-word tiles) are tuned;
    the trajectory equals the untuned one (fixed rule: 256-word tiles here), and a
    second plan of the same shape takes the cached choice without new trials."""
    Ls = [512, 512]
    betas = W.beta_grid(64, 0.3, 0.6, 64)
    seeds = [W.BASE_SEED + g for g in range(2)]
    S.shaken_autotune_clear()
    t0, _ = S.shaken_autotune_stats()
    b, ctxs = batch_of(S, Ls, betas, seeds, True)
    wpt = S.shaken_batch_lattice_wpt(b, S.MULTISPIN)
    assert wpt in (1, 4)
    t1, cached = S.shaken_autotune_stats()
    assert t1 == t0 + 1 and cached >= 1
    S.shaken_batch_step(b, 3, False)
    S.shaken_batch_sync(b)
    tuned = [S.shaken_get_spins(c, 32, 512 * 512) for c in ctxs]
    free_batch(S, b, ctxs)

    b, ctxs = batch_of(S, Ls, betas, seeds, False)
    assert S.shaken_batch_lattice_wpt(b, S.MULTISPIN) == 1
    S.shaken_batch_step(b, 3, False)
    S.shaken_batch_sync(b)
    for c, ref in zip(ctxs, tuned):
        assert np.array_equal(S.shaken_get_spins(c, 32, 512 * 512), ref)
    free_batch(S, b, ctxs)

    b, ctxs = batch_of(S, Ls, betas, seeds, True)
    assert S.shaken_batch_lattice_wpt(b, S.MULTISPIN) == wpt
    assert S.shaken_autotune_stats()[0] == t1  # cache hit, no new trials
    free_batch(S, b, ctxs)


def test_every_launch_shape_gives_the_same_trajectory(S):
    """The tuner's two knobs -- lane words per thread (1, 4) and resident blocks per SM
    (every block that fits, or fewer) -- change only how tiles are spread over blocks:
    pinned in each shape, a batch of uneven groups follows the same trajectory, equal to
    the oracle's at sampled groups; the tuner's own choice is one of these shapes."""
    Ls = [512, 256, 512, 64]
    betas = W.beta_grid(32 * len(Ls), 0.3, 0.6, 64)
    seeds = [W.BASE_SEED + 50 + g for g in range(len(Ls))]
    b, ctxs = batch_of(S, Ls, betas, seeds, True)
    wpt, bps = S.shaken_batch_lattice_shape(b, S.MULTISPIN)
    assert wpt in (1, 4) and bps >= 1
    free_batch(S, b, ctxs)
    results = []
    for w in (1, 4):
        for p in (1, 2):
            b, ctxs = batch_of(S, Ls, betas, seeds, True)
            S.shaken_batch_set_lattice_shape(b, S.MULTISPIN, w, p)
            assert S.shaken_batch_lattice_shape(b, S.MULTISPIN) == (w, p)
            S.shaken_batch_step(b, 4, False)
            S.shaken_batch_sync(b)
            results.append([S.shaken_get_spins(c, 32, int(L) * int(L)) for c, L in zip(ctxs, Ls)])
            with pytest.raises(S.ShakenError):
                S.shaken_batch_set_lattice_shape(b, S.MULTISPIN, 2, 1)
            free_batch(S, b, ctxs)
    for r in results[1:]:
        for a, ref in zip(r, results[0]):
            assert np.array_equal(a, ref)
    L = Ls[3]
    o = core.lattice_init(L, 32, seeds[3], core.MODE_MULTISPIN, 0)
    o, _ = core.lattice_run(o, 1.0, 1.0, 0.0, betas[96:128], seeds[3], 0, 4, core.MODE_MULTISPIN)
    assert np.array_equal(results[0][3].reshape(32, L, L), o)


def test_small_family_is_not_tuned(S):
    t0, _ = S.shaken_autotune_stats()
    ctx = S.shaken_init(lattice_problem(S, S.MULTISPIN, 64, 32, W.beta_grid(32)), 5)
    assert S.shaken_lattice_wpt(ctx) == 1
    assert S.shaken_autotune_stats()[0] == t0
    S.shaken_free(ctx)


def test_bench_workload_sampled_sites(S):
    """The batched workload in the launch configuration the bench times (one batch,
    tuned tile shape): one full step, sampled sites of every group checked against the
    oracle's single-site updates."""
    Ls = W.multispin_group_sizes(GROUPS, W.BASE_SEED, L_CHOICES)
    betas = W.beta_grid(GROUPS * 32, 0.3, 0.6, 64)
    seeds = [W.BASE_SEED + g for g in range(GROUPS)]
    b, ctxs = batch_of(S, Ls, betas, seeds, True)
    assert S.shaken_batch_lattice_wpt(b, S.MULTISPIN) in (1, 4)
    s0 = [S.shaken_get_spins(c, 32, int(L) * int(L)).reshape(32, int(L), int(L))
          for c, L in zip(ctxs, Ls)]
    S.shaken_batch_step(b, 1, False)
    S.shaken_batch_sync(b)
    g = np.random.default_rng(11)
    J, q, lam = 1.0, 1.0, 0.0
    for k, (c, L) in enumerate(zip(ctxs, Ls)):
        L = int(L)
        s1 = S.shaken_get_spins(c, 32, L * L).reshape(32, L, L)
        for _ in range(4):
            r = int(g.integers(32))
            i, j = int(g.integers(L)), int(g.integers(L))
            beta = float(betas[32 * k + r])
            loc = s0[k][r].copy()
            sp = {}
            for (a, bb) in ((i, j), ((i + 1) % L, j), (i, (j + 1) % L)):
                sp[(a, bb)] = core.lattice_site(loc, a, bb, J, q, lam, beta, seeds[k], 0, 0,
                                                core.MODE_MULTISPIN, r)
            for key, v in sp.items():
                loc[key] = v
            tau = core.lattice_site(loc, i, j, J, q, lam, beta, seeds[k], 0, 1,
                                    core.MODE_MULTISPIN, r)
            assert s1[r, i, j] == tau
    free_batch(S, b, ctxs)
