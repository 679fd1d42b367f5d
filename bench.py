#!/usr/bin/env python3
"""Throughput of the shaken-dynamics half-step update (arXiv:1904.06257) on GB300.

Workload (one "step" = one full shaken step P^dl then P^ur of every replica):
  batched multispin lattices -- 128 groups of 32 replicas (4096 replicas), each
  group an L x L periodic torus with L drawn uniformly from {32, 64, 128, 256,
  512}, J = 1, q = 1, lambda = 0, beta_r = 0.3 + 0.3 (r mod 64) / 63, random
  start, all groups stepped by one launch per half step.
Metric: site-updates/s (2 |V| R per step), whole job over all ranks.

Also reported: the plain single-lattice kernel (L = 4096, int8, one replica)
on the same GPU, end-to-end throughput through the public C ABI with host
buffers, the roofline of the dominant kernel and the CPU oracle baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1904_06257_gb300 import workloads as W  # noqa: E402

GROUPS = 128
REPLICAS_PER_GROUP = 32
L_CHOICES = (32, 64, 128, 256, 512)
Q, J, LAM = 1.0, 1.0, 0.0
FLUSH_BYTES = 256 << 20  # > 129 MB L2
# the half-step launches of every 4th timed step are bracketed by CUDA events: the
# events take device time themselves (about 4% of a step when every launch is timed)
TIMING_STRIDE = 4


def workload(rank: int):
    Ls = W.multispin_group_sizes(GROUPS, W.BASE_SEED, L_CHOICES)
    betas = W.beta_grid(GROUPS * REPLICAS_PER_GROUP, 0.3, 0.6, 64)
    seeds = [W.BASE_SEED + 100003 * rank + g for g in range(GROUPS)]
    return Ls, betas, seeds


def updates_per_step(Ls) -> float:
    return 2.0 * REPLICAS_PER_GROUP * float(np.sum(np.asarray(Ls, dtype=np.float64) ** 2))


def aggregate(updates_local: float, ms_local: float, world: int, device="cpu"):
    """Whole-job rate of ranks that each run their own groups (weak scaling, no exchange
    on the data path): the site updates of every rank, summed, over the slowest rank's
    time.  Returns (updates/s, slowest rank's ms)."""
    import torch
    upd = torch.tensor([float(updates_local)], dtype=torch.float64, device=device)
    ms = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(upd, op=torch.distributed.ReduceOp.SUM)
        torch.distributed.all_reduce(ms, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.barrier()
    return float(upd.item()) / (float(ms.item()) * 1e-3), float(ms.item())


# ------------------------------------------------------------------------ clocks
class Clocks:
    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------ oracle (CPU)
def _oracle_group(args):
    L, betas, seed, steps = args
    from oracle import core
    s = core.lattice_init(L, REPLICAS_PER_GROUP, seed, core.MODE_MULTISPIN, 0)
    t0 = time.perf_counter()
    core.lattice_run(s, J, Q, LAM, betas, seed, 0, steps, core.MODE_MULTISPIN)
    dt = time.perf_counter() - t0
    return 2.0 * REPLICAS_PER_GROUP * L * L * steps, dt


def _warm(_):
    from oracle import core  # noqa: F401
    return 0


def oracle_pool(n_groups):
    """A spawned process pool for the oracle (spawn: safe after CUDA is initialised)."""
    from oracle import core
    core.build()
    workers = max(1, min(n_groups, os.cpu_count() or 1))
    pool = mp.get_context("spawn").Pool(workers)
    pool.map(_warm, range(workers))
    return pool, workers


def oracle_sample_plan(Ls, per_size, max_L=None):
    """(L, group, full steps) of the oracle sample: the first `per_size` groups of each
    lattice size up to max_L (all sizes when None), each for round(top^2 / L^2) steps,
    top the largest size taken (about equal updates per group)."""
    sizes = sorted(set(int(x) for x in Ls if max_L is None or int(x) <= max_L))
    top = max(sizes) ** 2
    plan = []
    for L in sizes:
        steps = max(1, round(top / (L * L)))
        plan += [(L, g, steps) for g in range(len(Ls)) if int(Ls[g]) == L][:per_size]
    return plan


def oracle_sample(pool, workers, Ls, betas, seeds, per_size=3, max_L=None):
    """Run the CPU oracle, as it stands, on the first `per_size` groups of every
    lattice size of the workload up to max_L (32 replicas each), one task per group on
    the pool, each group for as many full steps as the largest size's one step is
    worth in updates (so the tasks take about the same time), and return (updates/s
    over the wall time, cores used, description, updates, wall)."""
    plan = oracle_sample_plan(Ls, per_size, max_L)
    top = max(L for L, _, _ in plan) ** 2
    jobs = [(L, betas[32 * g:32 * g + 32], seeds[g], steps) for L, g, steps in plan]
    workers = min(workers, len(jobs))
    t0 = time.perf_counter()
    res = pool.map(_oracle_group, jobs, chunksize=1)
    wall = time.perf_counter() - t0
    upd = sum(r[0] for r in res)
    per = ", ".join(f"L={L}: {st}" for L, st in sorted(set((L, st) for L, _, st in plan)))
    desc = (f"{len(jobs)} groups of the workload, {per_size} at each L "
            f"{'' if max_L is None else f'<= {max_L} '}(32 replicas each), full steps per "
            f"group {per} (about equal work per group), one spawned process per group")
    return upd / wall, workers, desc, upd, wall


def reference_max_L(n_samples: int):
    """Largest lattice size in the reference arm's per-step sample, so that n_samples
    samples end within a few minutes: a group's step at L = 512 takes ~7 s of one Grace
    core, at 256 ~1.7 s, at 128 ~0.4 s (the oracle's rate does not depend on L)."""
    if n_samples <= 30:
        return None
    return 256 if n_samples <= 100 else 128


def _oracle_config(task):
    """One bounded single-threaded oracle run of a configuration's workload:
    returns (name, updates, seconds, description)."""
    from oracle import core
    kind = task[0]
    if kind == "lattice":
        _, name, L, beta, q, steps = task
        s = core.lattice_init(L, 1, W.BASE_SEED, core.MODE_SINGLE, 0)
        t0 = time.perf_counter()
        core.lattice_run(s, 1.0, q, 0.0, beta, W.BASE_SEED, 0, steps, core.MODE_SINGLE)
        dt = time.perf_counter() - t0
        return name, 2.0 * L * L * steps, dt, f"L={L}, 1 replica, {steps} full step(s)"
    if kind == "multispin":
        _, name, L, steps = task
        betas = W.beta_grid(REPLICAS_PER_GROUP, 0.3, 0.6, 64)
        s = core.lattice_init(L, REPLICAS_PER_GROUP, W.BASE_SEED, core.MODE_MULTISPIN, 0)
        t0 = time.perf_counter()
        core.lattice_run(s, J, Q, LAM, betas, W.BASE_SEED, 0, steps, core.MODE_MULTISPIN)
        dt = time.perf_counter() - t0
        return name, 2.0 * REPLICAS_PER_GROUP * L * L * steps, dt, \
            f"one group of 32 replicas at L={L}, {steps} full step(s)"
    _, name, n, integer, R, steps = task
    u, v = W.erdos_renyi(n, 8.0, W.BASE_SEED + 1)
    Jc = (W.couplings_pm1(u.size, W.BASE_SEED + 2) if integer
          else W.couplings_normal(u.size, W.BASE_SEED + 2))
    lam = W.fields_normal(n, 0.1, W.BASE_SEED + 3)
    tail, head = core.orient(u, v, 0)
    s = core.graph_init(n, R, W.BASE_SEED)
    t0 = time.perf_counter()
    core.graph_run(s, tail, head, Jc, integer, lam, 1.0, 0.1, W.BASE_SEED, 0, steps,
                   draw=core.DRAW_PLANE if integer else core.DRAW_DIRECT)
    dt = time.perf_counter() - t0
    return name, 2.0 * n * R * steps, dt, \
        f"ER n={n}, mean degree 8, {'+-1' if integer else 'N(0,1)'} couplings, " \
        f"lambda ~ N(0, 0.1^2), {R} replicas, {steps} full step(s) at beta = 0.1"


def oracle_configs():
    """The oracle, as it stands, on bounded samples of each configuration (one
    single-threaded process per sample, the samples run side by side)."""
    tasks = [("lattice", "C1 L=64", 64, 0.40, 1.0, 500),
             ("lattice", "C2 L=4096", 4096, 0.4407, 1.0, 1)]
    tasks += [("multispin", f"C3 L={L}", L, 1) for L in (32, 64, 128, 256, 512)]
    # the +-1 graph oracle draws every lane's uniform from 32 bit planes (32 Philox calls
    # per update), hence the smaller sample
    tasks += [("graph", "C4 ER n=1e4 +-1", 10_000, True, 256, 1),
              ("graph", "C4 ER n=1e5 N(0,1)", 100_000, False, 256, 1)]
    pool, _ = oracle_pool(len(tasks))
    res = pool.map(_oracle_config, tasks)
    pool.close()
    pool.join()
    return {name: {"updates_per_s": upd / dt, "updates": upd, "seconds": dt, "sample": desc,
                   "cores": 1} for name, upd, dt, desc in res}


# ------------------------------------------------------------------------ GPU arm
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1904_06257_gb300 import build
    build.build()
    from paper_1904_06257_gb300 import shaken as S
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    if (args.only_graphs or args.only_serving or args.only_small or args.only_plain
            or args.only_config2):
        if rank == 0:
            if args.only_small:
                part = run_small(S, stream)
            elif args.only_config2:
                part = run_config2(S, stream, torch)
            elif args.only_plain:
                part = run_plain(S, stream, torch)
            elif args.only_graphs:
                part = run_graphs(S, stream, torch, args)
            else:
                part = run_serving(S, stream, args)
            print(json.dumps(part), flush=True)
        return None
    Ls, betas, seeds = workload(rank)
    ups = updates_per_step(Ls)

    # ---- batched multispin groups
    ctxs = []
    batch = S.shaken_batch_create(stream)
    for g in range(GROUPS):
        p = S.Problem(S.LATTICE, S.MULTISPIN, REPLICAS_PER_GROUP, betas[32 * g:32 * g + 32], Q,
                      L=int(Ls[g]), J=J, lambda_const=LAM)
        c = S.shaken_init(p, seeds[g], stream)
        S.shaken_batch_add(batch, c)
        ctxs.append(c)
    if args.no_autotune:  # fixed launch-shape rule (profiling runs: no timed trial launches)
        S.shaken_batch_set_autotune(batch, False)
    tile_wpt = S.shaken_batch_lattice_wpt(batch, S.MULTISPIN)  # autotuned launch shape
    # RNG accounting over two warm-up steps (not timed)
    counter = torch.zeros(1, dtype=torch.int64, device=dev)
    S.shaken_batch_set_rng_counter(batch, counter.data_ptr())
    S.shaken_batch_step(batch, 2, False)
    S.shaken_batch_sync(batch)
    calls_per_launch = float(counter.item()) / 4.0
    S.shaken_batch_set_rng_counter(batch, None)
    S.shaken_batch_step(batch, max(args.warmup, 3), False)
    S.shaken_batch_sync(batch)

    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    # clocks: sampled from a sustained ~1.5 s load right before the timed region
    # through its end (the timed region alone is shorter than the 200 ms sampling)
    clk = Clocks(local_rank)
    t_end = time.perf_counter() + 1.5
    while time.perf_counter() < t_end:
        S.shaken_batch_step(batch, 32, True)
        S.shaken_batch_sync(batch)
    S.shaken_batch_set_timing(batch, TIMING_STRIDE)
    l0 = S.shaken_batch_launch_count(batch)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            ev[k][0].record(stream)
        S.shaken_batch_step(batch, 1, False)
        with torch.cuda.stream(stream):
            ev[k][1].record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = S.shaken_batch_launch_count(batch) - l0
    step_ms = sum(a.elapsed_time(b) for a, b in ev)
    kern_ms, kern_n = S.shaken_batch_kernel_time(batch)
    S.shaken_batch_set_timing(batch, False)
    value, step_ms_max = aggregate(ups * args.steps, step_ms, world, dev)
    if args.only_batched:
        if rank == 0:
            print(json.dumps({"value": value, "unit": "updates/s", "steps": args.steps,
                              "kernel_ms_per_launch": kern_ms / max(kern_n, 1),
                              "calls_per_launch": calls_per_launch}), flush=True)
        return None

    # ---- CUDA-graph replay of the same batch (steady state, no flush): context
    S.shaken_batch_step(batch, 64, True)
    S.shaken_batch_sync(batch)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
    S.shaken_batch_step(batch, 128, True)
    with torch.cuda.stream(stream):
        e1.record(stream)
    stream.synchronize()
    graph_rate = ups * 128 / (e0.elapsed_time(e1) * 1e-3)

    # ---- unbatched: each group on its own (one launch sequence per group)
    for c in ctxs:
        S.shaken_batch_remove(batch, c)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nst = 4
    for c in ctxs:
        S.shaken_step(c, nst)
    for c in ctxs:
        S.shaken_sync(c)
    torch.cuda.synchronize()
    unbatched_rate = ups * nst / (time.perf_counter() - t0)
    for c in ctxs:
        S.shaken_batch_add(batch, c)

    # ---- e2e through the C ABI with host buffers: a job uploads every group's
    # state from pinned host memory, runs K steps, reads every state and the
    # observables back.
    tot_bytes = S.shaken_batch_state_bytes(batch)
    host_in = torch.empty(tot_bytes, dtype=torch.uint8, pin_memory=True)
    host_out = torch.empty(tot_bytes, dtype=torch.uint8, pin_memory=True)
    g = np.random.default_rng(5)
    host_in.numpy()[:] = g.integers(0, 256, size=tot_bytes, dtype=np.uint8)

    def e2e_job(steps):
        S.shaken_batch_set_states_raw(batch, host_in.data_ptr(), tot_bytes)
        S.shaken_batch_step(batch, steps, True)
        S.shaken_batch_get_states_raw_async(batch, host_out.data_ptr(), tot_bytes)
        return S.shaken_batch_observables(batch, GROUPS * REPLICAS_PER_GROUP)  # one sync

    e2e_job(1)  # first use sets up the batch's packed-copy buffers (not timed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    obs = e2e_job(args.steps)
    e2e_s = time.perf_counter() - t0
    obs_bytes = obs.nbytes
    e2e_value, _ = aggregate(ups * args.steps, e2e_s * 1e3, world, dev)
    e2e = {"value": e2e_value, "unit": "updates/s",
           "h2d_bytes_per_step": int(tot_bytes / args.steps),
           "d2h_bytes_per_step": int((tot_bytes + obs_bytes) / args.steps),
           "what": "per job of K steps: the raw states of all 128 groups H2D in one copy "
                   "from pinned memory, K batched steps (CUDA graph), all states D2H in one "
                   "copy and the observables of all 4096 replicas (one batched call); "
                   "wall clock",
           "note": "can exceed value: the steps replay a CUDA graph and the state stays in "
                   "L2 between them, while every device-timed step starts after an L2 "
                   "flush"}

    # ---- plain single-lattice kernel: L = 4096, one replica, int8 and bit-packed
    plain = run_plain(S, stream, torch)
    plain_rate = plain["int8"]

    # ---- plain-lattice sweep: L = 4096, lambda x q x beta x encoding x start, 2000 steps each
    config2 = None if args.skip_config2 else run_config2(S, stream, torch)

    # ---- small lattice: L = 64 int8, one replica, beta = 0.40, 10^4 steps with m and H per step
    small = run_small(S, stream)

    # ---- metastable regime (Sec. 3.2): m(t) from -1 at q = 0.1, lambda = 0.15
    meta = run_metastability(S, stream)

    # ---- arbitrary sparse graphs: n = 1e6, 256 replicas, lambda_x ~ N(0, 0.1^2), q = 1
    graphs = {} if args.skip_graphs else run_graphs(S, stream, torch, args)

    # ---- serving: Poisson stream of anneal jobs, continuous batching
    serving = None if args.skip_serving else run_serving(S, stream, args)

    # ---- roofline of the dominant kernel (multispin half step)
    rates = {name: S.shaken_microbench(k)[0] for k, name in enumerate(MICROBENCH_KINDS)}
    avg_kernel_s = (kern_ms / max(kern_n, 1)) * 1e-3
    traffic = committed_traffic("lattice_half_kernel<MULTISPIN>")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_ph = philox_peak_derived(sms)
    # the roofline's peak: Philox calls per second with the plane comparisons each call
    # feeds (4 planes x 4 logic operations), at the measured Philox and LOP3 rates, the
    # two kinds of work one after the other
    peak = 1.0 / (1.0 / rates["philox_calls"] + PLANE_OPS_PER_CALL / rates["lop3"])
    alg = (ups / 2.0) * ALG_CALLS_PER_UPDATE / avg_kernel_s  # algorithmic calls per second
    done = calls_per_launch / avg_kernel_s                   # calls actually made per second
    roofline = {"bound": "alu", "kernel": "lattice_half_kernel<MULTISPIN>",
                "achieved": done / 1e9, "peak": peak / 1e9,
                "unit": "G Philox-4x32-10 calls/s", "frac": done / peak,
                "traffic": traffic,
                "work": "Philox-4x32-10 calls the kernel makes (device counter): the bit-plane "
                        "comparison stops drawing once all 32 lanes of a word are decided",
                "peak_source": "measured on this GPU (shaken_microbench, all SMs): "
                               "1 / (1 / Philox calls/s + 16 / LOP3/s): each call with the "
                               "four planes it feeds, four logic operations per plane, the "
                               "two kinds of work not overlapped",
                "calls_per_launch": calls_per_launch,
                "frac_of_measured_philox": done / rates["philox_calls"],
                "philox_only": {"peak": peak_ph / 1e9, "frac": done / peak_ph,
                                "source": f"derived: {sms} SMs x {sm_max_mhz():.0f} MHz x "
                                          f"{WIDE_MUL_PER_CLK_PER_SM} wide multiplies/clk/SM / "
                                          f"{WIDE_MUL_PER_CALL} per call; no plane logic"},
                "calls_plus_planes": calls_plus_planes(calls_per_launch, avg_kernel_s, rates,
                                                       sms),
                "algorithmic": {"unit": "1/4 Philox-4x32-10 call per site update: one 32-bit "
                                        "uniform per decision, as the oracle draws it",
                                "achieved": alg / 1e9, "frac": alg / peak_ph,
                                "note": "above 1 because the kernel never needs most of those "
                                        "draws; not a roofline fraction"},
                "updates_per_launch": ups / 2.0,
                "avg_launch_ms": avg_kernel_s * 1e3,
                "timed_launches": kern_n,
                "timed_every_nth_step": TIMING_STRIDE,
                "microbench_per_s": rates,
                # HBM side: 0.25 B per update (one state bit read and written)
                "hbm_view": {
                    "achieved": (ups / 2.0) * 0.25 / avg_kernel_s / 1e9,
                    "peak": hbm_peak_gbs(), "unit": "GB/s",
                    "frac": ((ups / 2.0) * 0.25 / avg_kernel_s / 1e9) / hbm_peak_gbs()}}

    out = None
    if rank == 0:
        cpu = None
        if world == 1:
            pool, workers = oracle_pool(GROUPS)
            v, cores, desc, upd, wall = oracle_sample(pool, workers, Ls, betas, seeds, 3)
            pool.close()
            pool.join()
            cpu = {"value": v, "unit": "updates/s", "cores": cores, "kind": "oracle",
                   "sample": desc, "updates": upd, "wall_s": wall}
        out = {
            "metric": "site-updates/s (batched multispin shaken dynamics)",
            "value": value, "unit": "updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": "batched multispin: 128 groups x 32 replicas (4096), "
                                   "L uniform in {32,64,128,256,512}, beta grid of 64 in "
                                   "[0.3,0.6], J=1, q=1, lambda=0, periodic",
                       "L_per_group_sum_sq": int(np.sum(np.asarray(Ls) ** 2)),
                       "updates_per_step": ups, "replicas": GROUPS * REPLICAS_PER_GROUP,
                       "l2": "flushed between timed steps (256 MiB write outside the events)",
                       "parallelism": f"replicas/groups sharded over {world} GPU(s)",
                       "lane_words_per_thread": tile_wpt},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks,
            "graphs": graphs,
            "small_lattice": small,
            "config2": config2,
            "metastability": meta,
            "serving": serving,
            "batched_vs_plain": {
                "batched_updates_per_s": value / world,
                "batched_graph_replay_updates_per_s": graph_rate,
                "unbatched_same_groups_updates_per_s": unbatched_rate,
                "plain_int8_L4096_updates_per_s": plain_rate,
                "plain_packed_L4096_updates_per_s": plain["packed"]},
        }
    for c in ctxs:
        S.shaken_batch_remove(batch, c)
        S.shaken_free(c)
    S.shaken_batch_free(batch)
    return out


# ------------------------------------------------------------------------ traffic
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1904_06257_gb300", "csrc", f)
                  for f in ("lattice.cu", "shaken_internal.cuh")]


MICROBENCH_KINDS = ("philox_calls", "lop3", "imad", "lop3_imad_mix", "mad_wide", "mul_wide",
                    "mul_wide_lop3_mix", "philox_split_mul")
ALG_CALLS_PER_UPDATE = 0.25   # one 32-bit uniform per site update = 1/4 Philox-4x32-10 call
WIDE_MUL_PER_CLK_PER_SM = 32  # 32 x 32 -> 64-bit multiplies: 8 lanes/clk on each of 4 SMSPs
WIDE_MUL_PER_CALL = 20        # 10 rounds x 2
LOP3_PER_CLK_PER_SM = 64      # 32-bit logic operations: 16 lanes/clk on each of 4 SMSPs
SM_MAX_MHZ_FALLBACK = 2070.0


def sm_max_mhz() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        return SM_MAX_MHZ_FALLBACK


PLANE_OPS_PER_CALL = 16        # 4 planes x (select, complement, borrow, equality): mirror tables
LOP3_PER_CALL = 20             # 10 rounds x one three-input XOR for each of the two new words


def calls_plus_planes(calls: float, launch_s: float, rates: dict, sms: int) -> dict:
    """Launch-time bound of the multispin half step from the work it performs: the
    Philox calls it makes and the four logic operations per plane it compares for
    each call, the two kinds of work taken one after the other (no overlap).  Once
    with the measured rates of the microbenchmarks (Philox calls/s, LOP3/s), once
    with the rates the units allow (wide multiplies and LOP3 lanes per clock)."""
    meas = calls / rates["philox_calls"] + calls * PLANE_OPS_PER_CALL / rates["lop3"]
    clk = sms * sm_max_mhz() * 1e6
    unit = (calls * WIDE_MUL_PER_CALL / (WIDE_MUL_PER_CLK_PER_SM * clk)
            + calls * (LOP3_PER_CALL + PLANE_OPS_PER_CALL) / (LOP3_PER_CLK_PER_SM * clk))
    return {"plane_ops_per_call": PLANE_OPS_PER_CALL,
            "bound_ms_measured_rates": meas * 1e3, "frac_measured_rates": meas / launch_s,
            "bound_ms_unit_rates": unit * 1e3, "frac_unit_rates": unit / launch_s,
            "note": "bound = calls / Philox rate + 16 x calls / LOP3 rate (measured), or "
                    "20 wide multiplies per call at 32 lanes/clk/SM plus 36 logic operations "
                    "per call at 64 lanes/clk/SM (units); frac = bound / launch time"}


def philox_peak_derived(sms: int) -> float:
    """Philox-4x32-10 calls/s the wide-multiply units allow at the maximum SM clock."""
    return sms * sm_max_mhz() * 1e6 * WIDE_MUL_PER_CLK_PER_SM / WIDE_MUL_PER_CALL


def hbm_peak_gbs() -> float:
    """Measured copy bandwidth of this GPU model (MEASURED_PEAKS.json), else 6800."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from the
    committed ncu capture of `kernel`, or None when the kernel source changed since
    the capture (the record stores the source hash it was taken from)."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_hash") != kernel_source_hash():
        return None
    return rec.get("bytes_per_launch")


# ------------------------------------------------------------------------ plain lattice
def run_plain(S, stream, torch, L=4096, steps=512):
    """The plain single-lattice kernel: one L = 4096 replica (beta = 0.4407, q = J = 1,
    lambda = 0), int8 and bit-packed, `steps` full steps timed with CUDA events after
    a warm-up call of the same length (the banded kernel: one cooperative launch per
    call)."""
    plain = {}
    for name, enc in (("int8", S.INT8), ("packed", S.PACKED)):
        pp = S.Problem(S.LATTICE, enc, 1, 0.4407, Q, L=L, J=J, lambda_const=LAM)
        cp = S.shaken_init(pp, W.BASE_SEED + 7, stream)
        S.shaken_step(cp, steps)  # warm-up
        S.shaken_sync(cp)
        pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            pe0.record(stream)
        S.shaken_step(cp, steps)
        with torch.cuda.stream(stream):
            pe1.record(stream)
        stream.synchronize()
        plain[name] = 2.0 * L * L * steps / (pe0.elapsed_time(pe1) * 1e-3)
        S.shaken_free(cp)
    return plain


# ------------------------------------------------------------------------ plain-lattice sweep
C2_L, C2_STEPS, C2_BURN, C2_CHUNK = 4096, 2000, 1000, 50
C2_BETAS = (0.40, 0.4407, 0.48)
C2_QS = (0.5, 1.0, 2.0)
C2_ONSAGER_QS = (4.0, 8.0, 16.0)
REFERENCE_FILE = os.path.join(ROOT, "tests", "golden", "lattice_references.json")


def run_config2(S, stream, torch, L=C2_L, steps=C2_STEPS, burn=C2_BURN, chunk=C2_CHUNK):
    """The plain single-lattice sweep: L x L torus, J = 1, one replica, lambda in {0, 0.01},
    q in {0.5, 1, 2} (and q in {4, 8, 16} at lambda = 0 for the q -> infinity limit of
    Thm 3.1), beta in {0.40, 0.4407, 0.48}, int8 and bit-packed spins, all-plus and
    random starts, `steps` full steps each.  Per run: site-updates/s of the first
    `burn` steps (one stepping call, CUDA events), then the energy per site and |m|
    sampled every `chunk` steps over the rest.  At lambda = 0 they are compared with
    the exact stationary values of the shaken chain (the anisotropic triangular Ising
    measure it equals, tests/golden/lattice_references.json, written from the oracle's
    exact module): energy within 4 standard errors + 1e-3 wherever the run can reach
    equilibrium (not within 5% below or 3% above beta_c; from random starts only in the disordered
    phase), |m| < 5e-3 in the disordered phase from random starts (from +1 it decays
    over ~10^4 steps at large q) and within 4 standard errors + 2e-3 of
    the spontaneous magnetisation from the all-plus start in the ordered phase.  At
    lambda = 0.01 (no closed form) the magnetisation must exceed the lambda = 0 run's.
    Both encodings share seeds, so their trajectories (and observables) are identical.
    The q in {4, 8, 16} rows run int8 only and longer: an aligned spin flips with
    probability about e^{-2 beta (q - 2J)} per half step, so the run is `steps` times
    max(1, e^{2 beta (q - 4J)}) where that time scale is at most 1000 half steps; q = 16
    (e^{2 beta (q - 2J)} ~ 10^5 - 10^6) runs `steps` and is reported, not compared."""
    with open(REFERENCE_FILE) as f:
        refs = {(r["q"], r["beta"]): r for r in json.load(f)["points"]}
    cases = [(lam, q) for lam in (0.0, 0.01) for q in C2_QS] + [(0.0, q) for q in C2_ONSAGER_QS]
    runs, n_checked, failures = [], 0, []
    mags = {}
    idx = 0
    for lam, q in cases:
        extension = q in C2_ONSAGER_QS
        encs = (("int8", S.INT8),) if extension else (("int8", S.INT8), ("packed", S.PACKED))
        for beta in C2_BETAS:
            # an aligned spin flips with probability ~ e^{-2 beta (q - 2J)} per half step:
            # large q needs proportionally longer runs (q = 16 is out of reach)
            tau0 = math.exp(2.0 * beta * max(q - 2.0, 0.0))
            reachable = tau0 <= 1000.0
            n_steps = int(steps * max(1.0, math.exp(2.0 * beta * (q - 4.0)))) if reachable \
                else steps
            n_burn = n_steps - (steps - burn)
            for start in ("plus", "random"):
                seed = W.BASE_SEED + 4000 + idx
                idx += 1
                for name, enc in encs:
                    p = S.Problem(S.LATTICE, enc, 1, beta, q, L=L, J=1.0, lambda_const=lam,
                                  init=1 if start == "plus" else 0)
                    c = S.shaken_init(p, seed, stream)
                    dt = _timed(torch, stream, lambda: S.shaken_step(c, n_burn))
                    E, M = [], []
                    for _ in range((steps - burn) // chunk):
                        S.shaken_step(c, chunk)
                        o = S.shaken_observables(c, 1)
                        E.append(float(o["energy"][0]) / (L * L))
                        M.append(float(o["magnetization"][0]))
                    S.shaken_free(c)
                    E, M = np.array(E), np.array(M)
                    se_e = E.std(ddof=1) / math.sqrt(E.size)
                    se_m = np.abs(M).std(ddof=1) / math.sqrt(M.size)
                    row = {"enc": name, "lambda": lam, "q": q, "beta": beta, "start": start,
                           "steps": n_steps, "updates_per_s": 2.0 * L * L * n_burn / dt,
                           "energy_per_site": float(E.mean()), "energy_se": float(se_e),
                           "abs_m": float(np.abs(M).mean()), "m": float(M.mean()),
                           "abs_m_se": float(se_m)}
                    if lam == 0.0:
                        r = refs[(q, beta)]
                        bc = r["beta_c"]
                        ordered = beta > bc
                        # critical slowing down: within 5% below beta_c (3% above, where a
                        # run from +1 stays in its phase) 2000 steps do not equilibrate
                        near = (beta / bc - 1.0) < 0.03 if ordered else (1.0 - beta / bc) < 0.05
                        row.update({"energy_exact": r["energy_per_site"], "abs_m_exact": r["abs_m"],
                                    "beta_c": bc, "near_critical": near,
                                    "relaxation_reachable": reachable})
                        checks = []
                        ok_run = reachable and not near
                        if ok_run and (start == "plus" or not ordered):
                            checks.append(abs(E.mean() - r["energy_per_site"]) < 4 * se_e + 1e-3)
                        if ok_run and not ordered and start == "random":
                            checks.append(np.abs(M).mean() < 5e-3)
                        if ok_run and ordered and start == "plus":
                            checks.append(abs(np.abs(M).mean() - r["abs_m"]) < 4 * se_m + 2e-3)
                        row["compared"] = len(checks)
                        row["in_tolerance"] = bool(all(checks)) if checks else None
                        n_checked += len(checks)
                        if checks and not all(checks):
                            failures.append(row)
                    mags[(name, lam, q, beta, start)] = float(M.mean())
                    runs.append(row)
    order_ok = [mags[(n, 0.01, q, b, st)] > mags[(n, 0.0, q, b, st)]
                for (n, lam, q, b, st) in mags if lam == 0.0 and (n, 0.01, q, b, st) in mags]
    pairs = [(a, b) for a, b in zip(runs, runs[1:])
             if a["enc"] == "int8" and b["enc"] == "packed"
             and all(a[k] == b[k] for k in ("lambda", "q", "beta", "start"))]
    same = all(a["energy_per_site"] == b["energy_per_site"] and a["m"] == b["m"]
               for a, b in pairs)
    rates = {e: [r["updates_per_s"] for r in runs if r["enc"] == e] for e in ("int8", "packed")}
    return {"L": L, "steps": steps, "timed_steps": burn, "sample_every": chunk,
            "runs": runs, "checks": n_checked, "failures": len(failures),
            "lambda_0p01_raises_m": f"{sum(order_ok)}/{len(order_ok)}",
            "int8_equals_packed": bool(same), "int8_packed_pairs": len(pairs),
            "updates_per_s_median": {e: float(np.median(v)) for e, v in rates.items()},
            "updates_per_s_min": {e: float(np.min(v)) for e, v in rates.items()}}


# ------------------------------------------------------------------------ small lattice
def run_small(S, stream, L=64, steps=10000):
    """The small-lattice workload: L = 64 int8, one replica, beta = 0.40, q = J = 1,
    lambda = 0, 10^4 full steps with m and H of every step read back (one resident
    launch per 65536 steps)."""
    p1 = S.Problem(S.LATTICE, S.INT8, 1, 0.40, Q, L=L, J=J, lambda_const=LAM)
    c1 = S.shaken_init(p1, W.BASE_SEED, stream)
    S.shaken_step_record(c1, 100, 1)
    t0 = time.perf_counter()
    m1, e1 = S.shaken_step_record(c1, steps, 1)
    dt1 = time.perf_counter() - t0
    S.shaken_free(c1)
    return {"L": L, "steps": steps, "seconds": dt1,
            "updates_per_s": 2.0 * L * L * steps / dt1,
            "us_per_step": dt1 / steps * 1e6,
            "m_mean": float(m1[steps // 2:].mean()),
            "e_per_site_mean": float(e1[steps // 2:].mean() / L**2),
            "what": "shaken_step_record wall time: 10^4 steps with per-step m and H to host"}


# ------------------------------------------------------------------------ metastability
META_BETAS = (1.3, 2.3, 3.3, 4.0)


def run_metastability(S, stream, L=64, groups=4, steps=8000):
    """The shaken side of the paper's metastability runs (Sec. 3.2): J = 1, q = 0.1,
    lambda = 0.15, all replicas started at -1, m recorded every full step, for each
    beta of the paper's figure.  Reports m(t) averaged over the replicas at a few
    times, the first exit from -1, the tunnelling time (first step with m > 0) and
    the fraction of replicas that reached +1 itself."""
    out = {"L": L, "replicas": 32 * groups, "steps": steps, "J": 1.0, "q": 0.1,
           "lambda": 0.15, "betas": {}}
    marks = [t for t in (1, 10, 100, 1000, 4000, steps) if t <= steps]
    for beta in META_BETAS:
        mags = []
        for g in range(groups):
            p = S.Problem(S.LATTICE, S.MULTISPIN, 32, beta, 0.1, L=L, J=1.0, lambda_const=0.15,
                          init=2)
            c = S.shaken_init(p, W.BASE_SEED + 500 + g, stream)
            m, _ = S.shaken_step_record(c, steps, 32)
            S.shaken_free(c)
            mags.append(m)
        m = np.concatenate(mags, axis=1)  # [steps][replicas]
        out_ = m > -1.0
        first = np.where(out_.any(axis=0), out_.argmax(axis=0) + 1, -1)
        cross = m > 0.0  # in the + phase
        tun = np.where(cross.any(axis=0), cross.argmax(axis=0) + 1, -1)
        done = tun > 0
        out["betas"][str(beta)] = {
            "m_mean_at_step": {str(t): float(m[t - 1].mean()) for t in marks},
            "exit_from_minus_mean_steps": float(first[first > 0].mean()) if (first > 0).any()
            else None,
            "tunnelled_fraction": float(done.mean()),
            "tunnelling_median_steps": float(np.median(tun[done])) if done.any() else None,
            "all_plus_reached_fraction": float((m == 1.0).any(axis=0).mean()),
            "flip_probability_from_minus": 1.0 / (1.0 + math.exp(2 * beta * (2 + 0.1 - 0.15)))}
    return out


# ------------------------------------------------------------------------ graphs
GRAPH_N, GRAPH_R = 1_000_000, 256


def _timed(torch, stream, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
    fn()
    with torch.cuda.stream(stream):
        e1.record(stream)
    stream.synchronize()
    return e0.elapsed_time(e1) * 1e-3


def run_graphs(S, stream, torch, args):
    """Sparse-graph workloads: Erdos-Renyi (mean degree 8) with +-1 couplings -- the
    full linear anneal beta 0.1 -> 3.0 over 5000 steps, best energy and cut -- and
    throughput of the real-coupling path, of a random 3-regular graph and of a
    hub-heavy power-law graph, and the 2D Edwards-Anderson anneal.  args.graph_cases
    (comma-separated: anneal, real, reg3, powerlaw, ea2d) selects some of them."""
    cases = (set(args.graph_cases.split(",")) if getattr(args, "graph_cases", None)
             else {"anneal", "real", "reg3", "powerlaw", "ea2d"})
    out = {}
    n, R = GRAPH_N, GRAPH_R
    lam = W.fields_normal(n, 0.1, W.BASE_SEED + 3)
    steps = args.graph_anneal_steps
    k = 50
    if cases & {"anneal", "real"}:
        u, v = W.erdos_renyi(n, 8.0, W.BASE_SEED + 1)
    if "anneal" in cases:
        out["er_pm1_anneal"] = _graph_anneal(S, stream, torch, n, R, u, v, lam, steps)
    if "real" in cases:
        out["er_real_step"] = _graph_real(S, stream, torch, n, R, u, v, lam, k)
    if "reg3" in cases:
        out["reg3_pm1_step"] = _graph_reg3(S, stream, torch, n, R, lam, k)
    if "powerlaw" in cases:
        out["powerlaw_pm1_step"] = _graph_powerlaw(S, stream, torch, n, R, lam)
    if "ea2d" in cases:
        out["ea2d_pm1_anneal"] = _graph_ea2d(S, stream, torch, steps)
    return out


def _graph_anneal(S, stream, torch, n, R, u, v, lam, steps):
    """ER +-1 anneal beta 0.1 -> 3.0 with per-step best-energy tracking."""
    Jpm = W.couplings_pm1(u.size, W.BASE_SEED + 2)
    sched = W.linear_schedule(0.1, 3.0, steps)
    p = S.Problem(S.GRAPH, S.MULTISPIN, R, 0.1, 1.0, n=n, u=u, v=v, J_edge=Jpm,
                  J_is_integer=True, lambda_=lam)
    c = S.shaken_init(p, W.BASE_SEED + 11, stream)
    S.shaken_step(c, 2)
    S.shaken_sync(c)
    dt = _timed(torch, stream, lambda: S.shaken_anneal(c, sched))
    obs = S.shaken_observables(c, R)
    S.shaken_free(c)
    return {
        "n": n, "m": int(u.size), "replicas": R, "steps": steps,
        "updates_per_s": 2.0 * n * R * steps / dt, "seconds": dt,
        "best_energy_min": float(obs["best_energy"].min()),
        "best_energy_mean": float(obs["best_energy"].mean()),
        "final_energy_mean": float(obs["energy"].mean()),
        "cut_weight_best_replica": float(obs["cut_weight"][int(np.argmin(obs["energy"]))]),
        "cut_edges_best_replica": int(obs["cut_edges"][int(np.argmin(obs["energy"]))]),
        "note": "anneal with per-step best-energy tracking (fused into half 0)"}


def _graph_real(S, stream, torch, n, R, u, v, lam, k):
    """Real couplings N(0,1), fixed beta, throughput without tracking."""
    Jr = W.couplings_normal(u.size, W.BASE_SEED + 4)
    p = S.Problem(S.GRAPH, S.MULTISPIN, R, 1.0, 1.0, n=n, u=u, v=v, J_edge=Jr,
                  J_is_integer=False, lambda_=lam)
    c = S.shaken_init(p, W.BASE_SEED + 12, stream)
    S.shaken_step(c, 2)
    S.shaken_sync(c)
    dt = _timed(torch, stream, lambda: S.shaken_step(c, k))
    S.shaken_free(c)
    return {"updates_per_s": 2.0 * n * R * k / dt, "steps": k}


def _graph_reg3(S, stream, torch, n, R, lam, k):
    """+-1 on a random 3-regular graph, fixed beta."""
    u3, v3 = W.random_regular3(n, W.BASE_SEED + 5)
    J3 = W.couplings_pm1(u3.size, W.BASE_SEED + 6)
    p = S.Problem(S.GRAPH, S.MULTISPIN, R, 1.0, 1.0, n=n, u=u3, v=v3, J_edge=J3,
                  J_is_integer=True, lambda_=lam)
    c = S.shaken_init(p, W.BASE_SEED + 13, stream)
    S.shaken_step(c, 2)
    S.shaken_sync(c)
    dt = _timed(torch, stream, lambda: S.shaken_step(c, k))
    S.shaken_free(c)
    return {"updates_per_s": 2.0 * n * R * k / dt, "steps": k}


def _graph_powerlaw(S, stream, torch, n, R, lam):
    """+-1 on a hub-heavy power-law graph (Chung-Lu, exponent 2.1, mean degree 8): the
    vertices of degree above 255 go to the chunked hub kernel."""
    up, vp = W.power_law(n, 8.0, 2.1, W.BASE_SEED + 15)
    Jp = W.couplings_pm1(up.size, W.BASE_SEED + 16)
    deg = np.bincount(np.concatenate([up, vp]), minlength=n)
    indeg = np.bincount(vp, minlength=n)  # min -> max orientation: the larger id is the head
    outdeg = np.bincount(up, minlength=n)
    p = S.Problem(S.GRAPH, S.MULTISPIN, R, 1.0, 1.0, n=n, u=up, v=vp, J_edge=Jp,
                  J_is_integer=True, lambda_=lam)
    c = S.shaken_init(p, W.BASE_SEED + 15, stream)
    S.shaken_step(c, 2)
    S.shaken_sync(c)
    kp = 20
    dt = _timed(torch, stream, lambda: S.shaken_step(c, kp))
    S.shaken_free(c)
    return {
        "n": n, "m": int(up.size), "exponent": 2.1, "replicas": R, "steps": kp,
        "updates_per_s": 2.0 * n * R * kp / dt,
        "max_degree": int(deg.max()), "max_in_degree": int(indeg.max()),
        "max_out_degree": int(outdeg.max()),
        "hubs_in": int((indeg > 255).sum()), "hubs_out": int((outdeg > 255).sum()),
        "note": "vertices of degree above 255 in a half step's direction: the chunked hub "
                "kernel (one warp per 2048-edge chunk and group)"}


def _graph_ea2d(S, stream, torch, steps):
    """The optimisation use of Sec. 6 on a synthetic 2D Edwards-Anderson +-1 instance:
    L x L torus, couplings +-1 i.i.d., lambda = 0, q = 2.5 (> 2: the regime where the
    minimisers of the pair Hamiltonian carry over, Sec. 6), 256 replicas, linear anneal."""
    Le, Re, qe = 256, 256, 2.5
    ue, ve = W.lattice_as_graph(Le)
    Je = W.couplings_pm1(ue.size, W.BASE_SEED + 8)
    p = S.Problem(S.GRAPH, S.MULTISPIN, Re, 0.1, qe, n=Le * Le, u=ue, v=ve, J_edge=Je,
                  J_is_integer=True, orientation=S.ORIENT_GIVEN)
    c = S.shaken_init(p, W.BASE_SEED + 14, stream)
    sched = W.linear_schedule(0.1, 3.0, steps)
    S.shaken_step(c, 2)
    S.shaken_sync(c)
    dt = _timed(torch, stream, lambda: S.shaken_anneal(c, sched))
    obs = S.shaken_observables(c, Re)
    S.shaken_free(c)
    return {
        "L": Le, "q": qe, "replicas": Re, "steps": steps,
        "updates_per_s": 2.0 * Le * Le * Re * steps / dt, "seconds": dt,
        "best_energy_per_site_min": float(obs["best_energy"].min()) / (Le * Le),
        "best_energy_per_site_mean": float(obs["best_energy"].mean()) / (Le * Le),
        "note": "synthetic instance (the paper's EA instances are not published); energies "
                "per site of H(sigma) = -sum J s s over the best full-step configurations"}


# ------------------------------------------------------------------------ serving
def _serving_pool(args):
    """Pre-generated +-1 Erdos-Renyi graphs of the serving distribution (n log-uniform in
    [1e3, 1e6], mean degree uniform in [3, 16]); only the literal 200 jobs/s stream uses
    them (its thousands of jobs cannot each get a fresh graph in time)."""
    g = W.rng(W.BASE_SEED + 77)
    pool = []
    for k in range(args.serve_pool):
        n = int(round(np.exp(g.uniform(np.log(1e3), np.log(1e6)))))
        n += n % 2
        deg = float(g.uniform(3.0, 16.0))
        u, v = W.erdos_renyi(n, deg, W.BASE_SEED + 1000 + k)
        J = W.couplings_pm1(u.size, W.BASE_SEED + 2000 + k)
        pool.append((n, u, v, J))
    return pool


def _job_graph(jb):
    """A fresh +-1 Erdos-Renyi graph with the job's own n and mean degree."""
    u, v = W.erdos_renyi(jb["n"], jb["mean_degree"], jb["seed"] + 17)
    return jb["n"], u, v, W.couplings_pm1(u.size, jb["seed"] + 29)


def _serve(S, stream, jobs, graphs, args, step_scale, window_s=None, order=0):
    """Submit `jobs` at their arrival times (job k anneals graphs[k] -- or graphs[k mod
    len(graphs)] for a pool --, beta 0.1 -> 3.0), then drain -- or, with window_s, stop
    after window_s seconds and cancel what is left.  Latency = completion - arrival of
    the completed jobs.  The server admits by the device-memory budget and the work cap
    (site updates per step of the running set), in arrival order, first fit."""
    srv = S.shaken_server_create(int(args.serve_budget_gb * 2**30), 64, stream)
    S.shaken_server_set_policy(srv, args.serve_work_cap, order)
    t0 = time.perf_counter()
    ids, meta, lags = [], [], []
    for k, jb in enumerate(jobs):
        n, u, v, J = graphs[k % len(graphs)]
        steps = max(1, int(round(jb["steps"] * step_scale)))
        R = jb["replicas"]
        p = S.Problem(S.GRAPH, S.MULTISPIN, R, 0.1, 1.0, n=n, u=u, v=v, J_edge=J,
                      J_is_integer=True)
        delay = jb["arrival"] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        lags.append(max(0.0, -delay))
        ids.append(S.shaken_server_submit(srv, p, jb["seed"], W.linear_schedule(0.1, 3.0, steps)))
        meta.append((jb["arrival"], n, R, steps))
    if window_s is None:
        S.shaken_server_drain(srv, args.serve_timeout)
    else:
        rest = window_s - (time.perf_counter() - t0)
        if rest > 0:
            time.sleep(rest)
    wall = time.perf_counter() - t0
    upd, launches, done = S.shaken_server_stats(srv)
    queued, running = S.shaken_server_queue(srv)
    lat, states = [], [0, 0, 0]
    for jid, (arr, n, R, steps) in zip(ids, meta):
        st = S.shaken_server_poll(srv, jid)
        states[min(st, 2)] += 1
        if st == 2:
            _, ta, td = S.shaken_server_result(srv, jid, R)
            lat.append(td - arr)
    S.shaken_server_free(srv)
    work = sum(2.0 * n * R * st for _, n, R, st in meta)
    return {"jobs": len(ids), "completed": int(done), "queued_at_end": int(queued),
            "running_at_end": int(running), "wall_s": wall,
            "offered_updates": work, "served_updates_per_s": upd / wall,
            "latency_p50_s": float(np.percentile(lat, 50)) if lat else None,
            "latency_p99_s": float(np.percentile(lat, 99)) if lat else None,
            "latency_max_s": float(max(lat)) if lat else None,
            "submit_lag_max_s": float(max(lags) if lags else 0.0),
            "launches": int(launches)}


def run_serving(S, stream, args):
    """Continuous batching of annealing jobs through the server (Poisson arrivals of
    +-1 Erdos-Renyi anneals, n log-uniform in [1e3, 1e6], mean degree U[3, 16], a fresh
    graph per job, replicas log-uniform over multiples of 32 in [32, 1024], steps
    uniform in [1000, 20000] x step_scale):
    * capacity: a burst of jobs submitted at once, served updates/s over the makespan;
    * load sweep: Poisson streams at 50 / 70 / 90 % of that capacity -> p50 / p99
      latency (completion - arrival), every job drained to completion;
    * the literal stream (200 jobs/s, full step counts, pool graphs) for a fixed
      window: it offers hundreds of times the capacity, so the queue grows while the
      work cap keeps jobs completing; completions, queue depth and served rate are
      reported and the rest is cancelled."""
    scale = args.serve_step_scale
    out = {"step_scale": scale, "budget_gb": args.serve_budget_gb,
           "work_cap_updates_per_step": args.serve_work_cap, "admission": "arrival order, first fit",
           "graphs": "fresh per job (load sweep, capacity); literal stream: "
                     f"{args.serve_pool} pre-generated"}
    # expected work per job of the stream distribution (large sample, no GPU)
    sample = W.serving_stream(1000.0, 10.0, W.BASE_SEED + 9)
    mean_work = float(np.mean([2.0 * jb["n"] * jb["replicas"] *
                               max(1, int(round(jb["steps"] * scale))) for jb in sample]))
    # capacity
    burst = W.serving_stream(1000.0, 10.0, W.BASE_SEED + 4, max_jobs=args.serve_burst)
    for jb in burst:
        jb["arrival"] = 0.0
    cap = _serve(S, stream, burst, [_job_graph(jb) for jb in burst], args, scale)
    capacity = cap["offered_updates"] / cap["wall_s"]
    out["capacity"] = {"jobs": cap["jobs"], "makespan_s": cap["wall_s"],
                       "updates_per_s": capacity}
    # load sweep
    sweep = []
    for frac in (0.5, 0.7, 0.9):
        rate = frac * capacity / mean_work
        jobs = W.serving_stream(rate, args.serve_horizon, W.BASE_SEED + 3)
        r = _serve(S, stream, jobs, [_job_graph(jb) for jb in jobs], args, scale)
        r.update({"load": frac, "arrival_rate_per_s": rate, "horizon_s": args.serve_horizon,
                  "offered_updates_per_s": r["offered_updates"] / args.serve_horizon})
        sweep.append(r)
    out["load_sweep"] = sweep
    # literal stream
    pool = _serving_pool(args)
    lit = W.serving_stream(200.0, args.serve_literal_horizon, W.BASE_SEED + 3)
    # shortest total work first: under hundreds of times the capacity, the small jobs
    # (n log-uniform, so many of them) complete inside the window
    r = _serve(S, stream, lit, pool, args, 1.0, window_s=args.serve_literal_window, order=1)
    r.update({"admission": "shortest total work first", "arrival_rate_per_s": 200.0,
              "horizon_s": args.serve_literal_horizon,
              "window_s": args.serve_literal_window,
              "offered_updates_per_s": r["offered_updates"] / args.serve_literal_horizon})
    out["literal_stream"] = r
    # headline numbers: the 70 % load point
    mid = sweep[1]
    out.update({"latency_p50_s": mid["latency_p50_s"], "latency_p99_s": mid["latency_p99_s"],
                "served_updates_per_s": mid["served_updates_per_s"], "at_load": 0.7})
    return out


# ------------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return None
    Ls, betas, seeds = workload(0)
    tot_upd, tot_wall, cores, desc = 0.0, 0.0, 1, ""
    pool, workers = oracle_pool(16)
    for k in range(args.warmup + args.steps):
        v, cores, desc, upd, wall = oracle_sample(pool, workers, Ls, betas, seeds, 1,
                                                  reference_max_L(args.warmup + args.steps))
        if k >= args.warmup:
            tot_upd += upd
            tot_wall += wall
    pool.close()
    pool.join()
    val = tot_upd / tot_wall
    return {"impl": "reference", "metric": "site-updates/s (batched multispin shaken dynamics)",
            "value": val, "unit": "updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_wall * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "batched multispin: 128 groups x 32 replicas (4096), "
                                   "L uniform in {32,64,128,256,512}, beta grid of 64 in "
                                   "[0.3,0.6], J=1, q=1, lambda=0, periodic"},
            "cpu_baseline": {"value": val, "unit": "updates/s", "kind": "oracle", "cores": cores,
                             "sample": "each step: " + desc},
            "e2e": {"value": val, "unit": "updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--oracle-configs", action="store_true",
                    help="with --impl reference: time the oracle on a bounded sample of "
                         "every configuration instead")
    ap.add_argument("--only-batched", action="store_true",
                    help="time the batched workload only (profiling runs)")
    ap.add_argument("--skip-graphs", action="store_true", help="skip the sparse-graph section")
    ap.add_argument("--only-graphs", action="store_true",
                    help="run the sparse-graph section only (profiling runs)")
    ap.add_argument("--only-serving", action="store_true", help="run the serving section only")
    ap.add_argument("--only-small", action="store_true",
                    help="run the small-lattice section only (profiling runs)")
    ap.add_argument("--only-plain", action="store_true",
                    help="run the plain single-lattice section only (profiling runs)")
    ap.add_argument("--only-config2", action="store_true",
                    help="run the plain-lattice sweep (L = 4096) only")
    ap.add_argument("--skip-config2", action="store_true", help="skip the plain-lattice sweep")
    ap.add_argument("--no-autotune", action="store_true",
                    help="fixed lattice launch-shape rule instead of timed trials (profiling)")
    ap.add_argument("--graph-anneal-steps", type=int, default=5000)
    ap.add_argument("--graph-cases", default=None,
                    help="graph section: comma-separated subset of anneal, real, reg3, "
                         "powerlaw, ea2d (default: all)")
    ap.add_argument("--skip-serving", action="store_true")
    ap.add_argument("--serve-horizon", type=float, default=8.0,
                    help="seconds of arrivals of each load-sweep stream")
    ap.add_argument("--serve-burst", type=int, default=24, help="jobs of the capacity burst")
    ap.add_argument("--serve-literal-horizon", type=float, default=1.0,
                    help="seconds of arrivals of the literal 200 jobs/s stream")
    ap.add_argument("--serve-literal-window", type=float, default=8.0,
                    help="seconds the literal stream runs before the rest is cancelled")
    ap.add_argument("--serve-step-scale", type=float, default=0.05,
                    help="steps per job = U[1000, 20000] x this factor")
    ap.add_argument("--serve-pool", type=int, default=12, help="pre-generated graphs")
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--serve-work-cap", type=float, default=3e8,
                    help="site updates per step of the server's running set")
    ap.add_argument("--serve-timeout", type=float, default=120.0)
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference" and args.oracle_configs:
        out = {"impl": "reference", "oracle_configs": oracle_configs()} if rank == 0 else None
    elif args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl")
        out = run_ours(args, rank, world, local_rank)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
