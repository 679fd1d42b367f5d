"""Thin Python binding of libshaken (include/shaken.h): argument marshalling only.

Every function has the name of the C entry point it calls; all computation
happens in the CUDA library.  The library must have been built
(``paper_1904_06257_gb300.build.build()``); if it is missing, importing this
module raises -- there is no CPU fallback.

Streams: pass ``None`` (default stream), a ``torch.cuda.Stream`` or a raw
``cudaStream_t`` integer.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LATTICE, GRAPH = 0, 1
INT8, PACKED, MULTISPIN = 0, 1, 2
INIT_RANDOM, INIT_PLUS, INIT_MINUS, INIT_GIVEN = 0, 1, 2, 3
ORIENT_MIN_MAX, ORIENT_GIVEN = 0, 2
STATUS = {0: "ok", -1: "E_INVAL", -2: "E_NOMEM", -3: "E_CUDA", -4: "E_TIMEOUT", -5: "E_STATE",
          -6: "E_BUDGET"}


class ShakenError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class shaken_problem(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("encoding", ctypes.c_int32), ("L", ctypes.c_int64),
        ("boundary", ctypes.c_int32), ("frozen_mask", ctypes.c_void_p), ("n", ctypes.c_int64),
        ("m", ctypes.c_int64), ("u", ctypes.c_void_p), ("v", ctypes.c_void_p),
        ("J_edge", ctypes.c_void_p), ("J_is_integer", ctypes.c_int32),
        ("orientation", ctypes.c_int32), ("J", ctypes.c_double), ("lambda_", ctypes.c_void_p),
        ("lambda_const", ctypes.c_double), ("q", ctypes.c_double), ("replicas", ctypes.c_int32),
        ("beta", ctypes.c_void_p), ("init", ctypes.c_int32), ("init_spins", ctypes.c_void_p),
    ]


class shaken_obs(ctypes.Structure):
    _fields_ = [("magnetization", ctypes.c_double), ("energy", ctypes.c_double),
                ("pair_energy", ctypes.c_double), ("best_energy", ctypes.c_double),
                ("best_step", ctypes.c_int64), ("cut_edges", ctypes.c_int64),
                ("cut_weight", ctypes.c_double)]


OBS_DTYPE = np.dtype([("magnetization", "f8"), ("energy", "f8"), ("pair_energy", "f8"),
                      ("best_energy", "f8"), ("best_step", "i8"), ("cut_edges", "i8"),
                      ("cut_weight", "f8")])
assert OBS_DTYPE.itemsize == ctypes.sizeof(shaken_obs)


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libshaken.so is not built ({path}); run "
                          "paper_1904_06257_gb300.build.build() -- there is no CPU fallback")
    lib = ctypes.CDLL(path)
    vp, i32, i64, u64, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                             ctypes.c_size_t)
    d = ctypes.c_double
    sigs = {
        "shaken_init": [ctypes.POINTER(vp), ctypes.POINTER(shaken_problem), u64, vp],
        "shaken_step": [vp, u64],
        "shaken_anneal": [vp, vp, u64],
        "shaken_set_tracking": [vp, ctypes.c_int],
        "shaken_set_order": [vp, ctypes.c_int],
        "shaken_step_record": [vp, u64, vp, vp],
        "shaken_observables": [vp, vp],
        "shaken_get_spins": [vp, vp],
        "shaken_get_spins_prime": [vp, vp],
        "shaken_set_spins": [vp, vp],
        "shaken_get_step": [vp, ctypes.POINTER(u64)],
        "shaken_save": [vp, vp, ctypes.POINTER(sz)],
        "shaken_load": [vp, vp, sz],
        "shaken_debug_fields": [vp, ctypes.c_int, vp],
        "shaken_debug_exact_always": [vp, ctypes.c_int],
        "shaken_debug_band_stall": [vp],
        "shaken_debug_band_hurry": [vp, ctypes.c_int],
        "shaken_launch_count": [vp, ctypes.POINTER(u64)],
        "shaken_sync": [vp],
        "shaken_batch_create": [ctypes.POINTER(vp), vp],
        "shaken_batch_add": [vp, vp],
        "shaken_batch_remove": [vp, vp],
        "shaken_batch_step": [vp, u64, ctypes.c_int],
        "shaken_batch_sync": [vp],
        "shaken_batch_launch_count": [vp, ctypes.POINTER(u64)],
        "shaken_batch_set_timing": [vp, ctypes.c_int],
        "shaken_batch_kernel_time": [vp, ctypes.POINTER(d), ctypes.POINTER(u64)],
        "shaken_batch_set_rng_counter": [vp, vp],
        "shaken_batch_set_autotune": [vp, ctypes.c_int],
        "shaken_set_autotune": [vp, ctypes.c_int],
        "shaken_batch_lattice_wpt": [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
        "shaken_batch_lattice_shape": [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int)],
        "shaken_batch_set_lattice_shape": [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int],
        "shaken_lattice_wpt": [vp, ctypes.POINTER(ctypes.c_int)],
        "shaken_autotune_stats": [ctypes.POINTER(u64), ctypes.POINTER(u64)],
        "shaken_autotune_clear": [],
        "shaken_microbench": [ctypes.c_int, ctypes.POINTER(d), ctypes.POINTER(d)],
        "shaken_state_bytes": [vp, ctypes.POINTER(sz)],
        "shaken_set_state_raw": [vp, vp, sz],
        "shaken_get_state_raw": [vp, vp, sz],
        "shaken_get_state_raw_async": [vp, vp, sz],
        "shaken_batch_observables": [vp, vp],
        "shaken_batch_state_bytes": [vp, ctypes.POINTER(sz)],
        "shaken_batch_set_states_raw": [vp, vp, sz],
        "shaken_batch_get_states_raw_async": [vp, vp, sz],
        "shaken_server_create": [ctypes.POINTER(vp), sz, ctypes.c_uint32, vp],
        "shaken_server_submit": [vp, ctypes.POINTER(shaken_problem), u64, vp, u64,
                                 ctypes.POINTER(i64)],
        "shaken_server_poll": [vp, i64, ctypes.POINTER(ctypes.c_int)],
        "shaken_server_set_policy": [vp, d, ctypes.c_int, ctypes.c_int],
        "shaken_server_queue": [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)],
        "shaken_server_result_state": [vp, i64, vp, sz],
        "shaken_server_result": [vp, i64, vp, ctypes.POINTER(d), ctypes.POINTER(d)],
        "shaken_server_drain": [vp, d],
        "shaken_server_stats": [vp, ctypes.POINTER(d), ctypes.POINTER(u64), ctypes.POINTER(i64)],
        "shaken_philox_device": [u64, vp, vp, i64, vp],
        "shaken_lattice_observables_noalloc": [vp, vp, i32, i64, i32, d, d, d, vp, vp],
        "shaken_threshold_device": [vp, vp, vp, i64, vp],
    }
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    for name in ("shaken_free", "shaken_batch_free", "shaken_server_free"):
        getattr(lib, name).argtypes = [vp]
        getattr(lib, name).restype = None
    for name in ("shaken_strerror",):
        getattr(lib, name).argtypes = [ctypes.c_int]
        getattr(lib, name).restype = ctypes.c_char_p
    for name in ("shaken_last_error", "shaken_version"):
        getattr(lib, name).argtypes = []
        getattr(lib, name).restype = ctypes.c_char_p
    return lib


_lib = _load()
LIB_PATH = _build.LIB


def _check(st: int):
    if st != 0:
        raise ShakenError(st, _lib.shaken_last_error().decode())


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(int(s.cuda_stream))
    return ctypes.c_void_p(int(s))


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


class Problem:
    """Owns the numpy arrays behind a ``shaken_problem`` struct."""

    def __init__(self, kind, encoding, replicas, beta, q, *, L=0, J=1.0, lambda_const=0.0,
                 lambda_=None, boundary=0, frozen_mask=None, n=0, u=None, v=None, J_edge=None,
                 J_is_integer=False, orientation=ORIENT_MIN_MAX, init=INIT_RANDOM,
                 init_spins=None):
        self._keep = []

        def arr(x, dt):
            if x is None:
                return None
            a = np.ascontiguousarray(x, dtype=dt)
            self._keep.append(a)
            return a

        b = arr(np.broadcast_to(np.asarray(beta, dtype=np.float64), (replicas,)), np.float64)
        self.replicas = replicas
        self.kind = kind
        self.sites = L * L if kind == LATTICE else n
        s = shaken_problem()
        s.kind, s.encoding, s.L, s.boundary = kind, encoding, L, boundary
        s.frozen_mask = _ptr(arr(frozen_mask, np.uint8))
        uu, vv, jj = arr(u, np.int32), arr(v, np.int32), arr(J_edge, np.float32)
        s.n = n
        s.m = 0 if uu is None else uu.size
        s.u, s.v, s.J_edge = _ptr(uu), _ptr(vv), _ptr(jj)
        s.J_is_integer = int(bool(J_is_integer))
        s.orientation = orientation
        s.J = J
        s.lambda_ = _ptr(arr(lambda_, np.float32))
        s.lambda_const = lambda_const
        s.q = q
        s.replicas = replicas
        s.beta = _ptr(b)
        s.init = init
        s.init_spins = _ptr(arr(init_spins, np.int8))
        self.struct = s


# --------------------------------------------------------------------------- contexts
def shaken_init(problem: Problem, seed: int, stream=None):
    ctx = ctypes.c_void_p()
    _check(_lib.shaken_init(ctypes.byref(ctx), ctypes.byref(problem.struct), seed,
                            _stream(stream)))
    return ctx


def shaken_free(ctx):
    _lib.shaken_free(ctx)


def shaken_step(ctx, n_steps: int):
    _check(_lib.shaken_step(ctx, n_steps))


def shaken_anneal(ctx, beta_schedule):
    b = np.ascontiguousarray(beta_schedule, dtype=np.float64)
    _check(_lib.shaken_anneal(ctx, _ptr(b), b.size))


def shaken_set_order(ctx, reversed_: bool):
    _check(_lib.shaken_set_order(ctx, int(bool(reversed_))))


def shaken_set_tracking(ctx, enable: bool):
    _check(_lib.shaken_set_tracking(ctx, int(bool(enable))))


def shaken_step_record(ctx, n_steps: int, replicas: int):
    mag = np.zeros((n_steps, replicas), dtype=np.float64)
    en = np.zeros((n_steps, replicas), dtype=np.float64)
    _check(_lib.shaken_step_record(ctx, n_steps, _ptr(mag), _ptr(en)))
    return mag, en


def shaken_observables(ctx, replicas: int):
    out = np.zeros(replicas, dtype=OBS_DTYPE)
    _check(_lib.shaken_observables(ctx, _ptr(out)))
    return out


def shaken_get_spins(ctx, replicas: int, sites: int):
    out = np.zeros((replicas, sites), dtype=np.int8)
    _check(_lib.shaken_get_spins(ctx, _ptr(out)))
    return out


def shaken_get_spins_prime(ctx, replicas: int, sites: int):
    out = np.zeros((replicas, sites), dtype=np.int8)
    _check(_lib.shaken_get_spins_prime(ctx, _ptr(out)))
    return out


def shaken_set_spins(ctx, spins):
    s = np.ascontiguousarray(spins, dtype=np.int8)
    _check(_lib.shaken_set_spins(ctx, _ptr(s)))


def shaken_get_step(ctx) -> int:
    t = ctypes.c_uint64()
    _check(_lib.shaken_get_step(ctx, ctypes.byref(t)))
    return t.value


def shaken_save(ctx) -> bytes:
    n = ctypes.c_size_t()
    _check(_lib.shaken_save(ctx, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(_lib.shaken_save(ctx, buf, ctypes.byref(n)))
    return buf.raw[: n.value]


def shaken_load(ctx, data: bytes):
    buf = ctypes.create_string_buffer(data, len(data))
    _check(_lib.shaken_load(ctx, buf, len(data)))


def shaken_debug_fields(ctx, half: int, replicas: int, sites: int):
    out = np.zeros((replicas, sites), dtype=np.float32)
    _check(_lib.shaken_debug_fields(ctx, half, _ptr(out)))
    return out


def shaken_debug_exact_always(ctx, on: bool):
    _check(_lib.shaken_debug_exact_always(ctx, int(bool(on))))


def shaken_debug_band_stall(ctx):
    """The next banded chunk's grid barrier never completes (timeout-path test)."""
    _check(_lib.shaken_debug_band_stall(ctx))


def shaken_debug_band_hurry(ctx, block: int):
    _check(_lib.shaken_debug_band_hurry(ctx, int(block)))


def shaken_launch_count(ctx) -> int:
    c = ctypes.c_uint64()
    _check(_lib.shaken_launch_count(ctx, ctypes.byref(c)))
    return c.value


def shaken_sync(ctx):
    _check(_lib.shaken_sync(ctx))


# --------------------------------------------------------------------------- batches
def shaken_batch_create(stream=None):
    b = ctypes.c_void_p()
    _check(_lib.shaken_batch_create(ctypes.byref(b), _stream(stream)))
    return b


def shaken_batch_add(batch, ctx):
    _check(_lib.shaken_batch_add(batch, ctx))


def shaken_batch_remove(batch, ctx):
    _check(_lib.shaken_batch_remove(batch, ctx))


def shaken_batch_step(batch, n_steps: int, use_graph: bool = True):
    _check(_lib.shaken_batch_step(batch, n_steps, int(bool(use_graph))))


def shaken_batch_sync(batch):
    _check(_lib.shaken_batch_sync(batch))


def shaken_batch_launch_count(batch) -> int:
    c = ctypes.c_uint64()
    _check(_lib.shaken_batch_launch_count(batch, ctypes.byref(c)))
    return c.value


def shaken_batch_set_autotune(batch, on: bool):
    _check(_lib.shaken_batch_set_autotune(batch, int(bool(on))))


def shaken_set_autotune(ctx, on: bool):
    _check(_lib.shaken_set_autotune(ctx, int(bool(on))))


def shaken_batch_set_lattice_shape(b, encoding: int, words_per_thread: int, blocks_per_sm: int):
    _check(_lib.shaken_batch_set_lattice_shape(b, int(encoding), int(words_per_thread),
                                               int(blocks_per_sm)))


def shaken_batch_lattice_shape(b, encoding: int):
    w, p = ctypes.c_int(), ctypes.c_int()
    _check(_lib.shaken_batch_lattice_shape(b, int(encoding), ctypes.byref(w), ctypes.byref(p)))
    return w.value, p.value


def shaken_batch_lattice_wpt(batch, encoding: int) -> int:
    v = ctypes.c_int()
    _check(_lib.shaken_batch_lattice_wpt(batch, int(encoding), ctypes.byref(v)))
    return v.value


def shaken_lattice_wpt(ctx) -> int:
    v = ctypes.c_int()
    _check(_lib.shaken_lattice_wpt(ctx, ctypes.byref(v)))
    return v.value


def shaken_autotune_stats():
    t, c = ctypes.c_uint64(), ctypes.c_uint64()
    _check(_lib.shaken_autotune_stats(ctypes.byref(t), ctypes.byref(c)))
    return t.value, c.value


def shaken_autotune_clear():
    _check(_lib.shaken_autotune_clear())


def shaken_batch_set_timing(batch, every):
    """every: 0 off, n > 0 time the half-step launches of every n-th step (True = 1)."""
    _check(_lib.shaken_batch_set_timing(batch, int(every)))


def shaken_batch_kernel_time(batch):
    ms, n = ctypes.c_double(), ctypes.c_uint64()
    _check(_lib.shaken_batch_kernel_time(batch, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def shaken_batch_set_rng_counter(batch, device_counter_ptr):
    _check(_lib.shaken_batch_set_rng_counter(
        batch, None if device_counter_ptr is None else ctypes.c_void_p(device_counter_ptr)))


def shaken_microbench(kind: int):
    r, ms = ctypes.c_double(), ctypes.c_double()
    _check(_lib.shaken_microbench(kind, ctypes.byref(r), ctypes.byref(ms)))
    return r.value, ms.value


def shaken_state_bytes(ctx) -> int:
    n = ctypes.c_size_t()
    _check(_lib.shaken_state_bytes(ctx, ctypes.byref(n)))
    return n.value


def shaken_set_state_raw(ctx, host_buf_ptr: int, nbytes: int):
    """host_buf_ptr: address of host memory (pinned for a fast copy) in the device encoding."""
    _check(_lib.shaken_set_state_raw(ctx, ctypes.c_void_p(host_buf_ptr), nbytes))


def shaken_get_state_raw(ctx, host_buf_ptr: int, nbytes: int):
    _check(_lib.shaken_get_state_raw(ctx, ctypes.c_void_p(host_buf_ptr), nbytes))


def shaken_get_state_raw_async(ctx, host_buf_ptr: int, nbytes: int):
    """Enqueue the copy of sigma; the buffer holds it after the next synchronising call."""
    _check(_lib.shaken_get_state_raw_async(ctx, ctypes.c_void_p(host_buf_ptr), nbytes))


def shaken_batch_state_bytes(batch) -> int:
    n = ctypes.c_size_t()
    _check(_lib.shaken_batch_state_bytes(batch, ctypes.byref(n)))
    return n.value


def shaken_batch_set_states_raw(batch, host_buf_ptr: int, nbytes: int):
    """All members' raw states (concatenated in member order) in one host-to-device copy."""
    _check(_lib.shaken_batch_set_states_raw(batch, ctypes.c_void_p(host_buf_ptr), nbytes))


def shaken_batch_get_states_raw_async(batch, host_buf_ptr: int, nbytes: int):
    """Enqueue the gather and one device-to-host copy of all members' states."""
    _check(_lib.shaken_batch_get_states_raw_async(batch, ctypes.c_void_p(host_buf_ptr), nbytes))


def shaken_batch_observables(batch, replicas_total: int):
    """Observables of every member's replicas, members in the order they were added."""
    out = np.zeros(replicas_total, dtype=OBS_DTYPE)
    _check(_lib.shaken_batch_observables(batch, _ptr(out)))
    return out


def shaken_batch_free(batch):
    _lib.shaken_batch_free(batch)


# --------------------------------------------------------------------------- server
def shaken_server_create(hbm_budget_bytes: int, chunk_steps: int = 64, stream=None):
    s = ctypes.c_void_p()
    _check(_lib.shaken_server_create(ctypes.byref(s), hbm_budget_bytes, chunk_steps,
                                     _stream(stream)))
    return s


def shaken_server_submit(server, problem: Problem, seed: int, beta_schedule) -> int:
    b = np.ascontiguousarray(beta_schedule, dtype=np.float64)
    jid = ctypes.c_int64()
    _check(_lib.shaken_server_submit(server, ctypes.byref(problem.struct), seed, _ptr(b), b.size,
                                     ctypes.byref(jid)))
    return jid.value


def shaken_server_poll(server, job_id: int) -> int:
    st = ctypes.c_int()
    _check(_lib.shaken_server_poll(server, job_id, ctypes.byref(st)))
    return st.value


def shaken_server_set_policy(server, max_step_updates: float = 3e8, order: int = 0,
                             keep_states: bool = False):
    _check(_lib.shaken_server_set_policy(server, float(max_step_updates), int(order),
                                         int(bool(keep_states))))


def shaken_server_queue(server):
    q, r = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.shaken_server_queue(server, ctypes.byref(q), ctypes.byref(r)))
    return q.value, r.value


def shaken_server_result_state(server, job_id: int, nbytes: int):
    out = np.zeros(nbytes, dtype=np.uint8)
    _check(_lib.shaken_server_result_state(server, job_id, _ptr(out), nbytes))
    return out


def shaken_server_result(server, job_id: int, replicas: int):
    out = np.zeros(replicas, dtype=OBS_DTYPE)
    ta, td = ctypes.c_double(), ctypes.c_double()
    _check(_lib.shaken_server_result(server, job_id, _ptr(out), ctypes.byref(ta),
                                     ctypes.byref(td)))
    return out, ta.value, td.value


def shaken_server_drain(server, timeout_s: float):
    _check(_lib.shaken_server_drain(server, timeout_s))


def shaken_server_stats(server):
    u, n, j = ctypes.c_double(), ctypes.c_uint64(), ctypes.c_int64()
    _check(_lib.shaken_server_stats(server, ctypes.byref(u), ctypes.byref(n), ctypes.byref(j)))
    return u.value, n.value, j.value


def shaken_server_free(server):
    _lib.shaken_server_free(server)


# --------------------------------------------------------------------------- primitives
def shaken_philox_device(seed: int, ctr_dev_ptr: int, out_dev_ptr: int, n: int, stream=None):
    _check(_lib.shaken_philox_device(seed, ctypes.c_void_p(ctr_dev_ptr),
                                     ctypes.c_void_p(out_dev_ptr), n, _stream(stream)))


def shaken_threshold_device(h_dev_ptr: int, beta_dev_ptr: int, out_dev_ptr: int, n: int,
                            stream=None):
    _check(_lib.shaken_threshold_device(ctypes.c_void_p(h_dev_ptr), ctypes.c_void_p(beta_dev_ptr),
                                        ctypes.c_void_p(out_dev_ptr), n, _stream(stream)))


def shaken_lattice_observables_noalloc(sigma_dev_ptr: int, sigma_prime_dev_ptr: int,
                                       encoding: int, L: int, replicas: int, J: float, q: float,
                                       lambda_const: float, stream=None):
    """Observables of caller-held device spin buffers; the library allocates nothing."""
    out = np.zeros(replicas, dtype=OBS_DTYPE)
    _check(_lib.shaken_lattice_observables_noalloc(
        ctypes.c_void_p(sigma_dev_ptr), ctypes.c_void_p(sigma_prime_dev_ptr), encoding, L,
        replicas, J, q, lambda_const, _ptr(out), _stream(stream)))
    return out


def shaken_version() -> str:
    return _lib.shaken_version().decode()
