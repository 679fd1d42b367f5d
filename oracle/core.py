"""ctypes wrapper of the plain-C oracle ``shaken_oracle.c``.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).  Every function here calls
one routine of the C file; the arithmetic lives there, one site at a time.
The library is compiled on first use (gcc, ``-O2 -ffp-contract=off``) into
``oracle/_build/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "shaken_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

INIT_STEP = 0xFFFFFFFF
MODE_SINGLE = 0  # lane word = 32 consecutive sites of one replica (int8, packed)
MODE_MULTISPIN = 1  # lane word = one site of 32 consecutive replicas
DRAW_DIRECT = 0  # graph lane k draws u_k = W_k
DRAW_PLANE = 1  # graph lane k draws its bits from the 32 words W_j (bit k of W_j = bit 31-j)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain C, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-shared",
               "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _i8p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))


def _u8p(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _f64p(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            _LIB = _open(build())
    return _LIB


def build_variant(source: str, tag: str) -> str:
    """Compile a modified copy of the oracle source (the planted-mistake tests) into
    ``oracle/_build/liboracle_<tag>.so`` with the flags of ``build``."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_BUILD, f"variant_{tag}.c")
    so = os.path.join(_BUILD, f"liboracle_{tag}.so")
    with open(src, "w") as f:
        f.write(source)
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-shared", "-fPIC",
           "-o", so, src, "-lm"]
    subprocess.run(cmd, check=True)
    return so


class using:
    """Context manager: every wrapper below calls the library at `path` instead."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _LIB
        lib()
        with _LOCK:
            self.saved = _LIB
            _LIB = _open(self.path)
        return self

    def __exit__(self, *exc):
        global _LIB
        with _LOCK:
            _LIB = self.saved
        return False


def _open(path: str):
    L = ctypes.CDLL(path)
    u32, u64, i64, d = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_double
    vp = ctypes.c_void_p
    L.orc_philox.argtypes = [vp, vp, vp]
    L.orc_exp.argtypes = [d]
    L.orc_exp.restype = d
    L.orc_threshold.argtypes = [d, d]
    L.orc_threshold.restype = u64
    L.orc_field.argtypes = [d, i64, d, ctypes.c_int, d]
    L.orc_field.restype = d
    L.orc_draw_plane.argtypes = [u64, u32, u32, u32, u32, ctypes.c_int]
    L.orc_draw_plane.restype = u32
    L.orc_draw_direct.argtypes = [u64, u32, u32, u32, u32, ctypes.c_int]
    L.orc_draw_direct.restype = u32
    L.orc_lattice_init.argtypes = [vp, i64, i64, vp, u64, ctypes.c_int, ctypes.c_int]
    L.orc_lattice_site.argtypes = [vp, i64, i64, i64, vp, d, d, d, d, u64, u32,
                                   ctypes.c_int, ctypes.c_int, i64]
    L.orc_lattice_site.restype = ctypes.c_int
    L.orc_lattice_half.argtypes = [vp, vp, i64, i64, vp, d, d, d, vp, u64, u32,
                                   ctypes.c_int, ctypes.c_int]
    L.orc_lattice_run.argtypes = [vp, vp, i64, i64, vp, d, d, d, vp, u64, u32, i64,
                                  ctypes.c_int]
    L.orc_lattice_anneal.argtypes = [vp, vp, i64, i64, vp, d, d, d, vp, u64, u32, i64,
                                     ctypes.c_int]
    L.orc_lattice_sums.argtypes = [vp, vp, i64, vp]
    L.orc_orient.argtypes = [i64, vp, vp, ctypes.c_int, vp, vp]
    L.orc_graph_half.argtypes = [vp, vp, i64, i64, vp, vp, vp, ctypes.c_int, vp, vp, d,
                                 vp, i64, u64, u32, ctypes.c_int, ctypes.c_int]
    L.orc_incidence.argtypes = [i64, i64, vp, vp, ctypes.c_int, vp, vp]
    L.orc_graph_field.argtypes = [vp, i64, vp, vp, vp, vp, vp, ctypes.c_int, vp, d,
                                  ctypes.c_int]
    L.orc_graph_field.restype = d
    L.orc_graph_draw.argtypes = [u64, i64, i64, u32, ctypes.c_int, ctypes.c_int]
    L.orc_graph_draw.restype = u32
    L.orc_graph_draws.argtypes = [vp, i64, i64, u64, u32, ctypes.c_int, ctypes.c_int]
    L.orc_graph_site.argtypes = [vp, i64, vp, vp, vp, vp, vp, ctypes.c_int, vp, vp, d, d,
                                 u64, u32, ctypes.c_int, ctypes.c_int, i64]
    L.orc_graph_site.restype = ctypes.c_int
    L.orc_graph_fields.argtypes = [vp, vp, i64, i64, vp, vp, vp, ctypes.c_int, vp, d, i64,
                                   ctypes.c_int]
    L.orc_graph_init.argtypes = [vp, i64, i64, vp, u64, ctypes.c_int]
    L.orc_graph_run.argtypes = [vp, vp, i64, i64, vp, vp, vp, ctypes.c_int, vp, vp, d,
                                vp, vp, i64, u64, u32, i64, ctypes.c_int]
    L.orc_graph_sums.argtypes = [vp, vp, i64, i64, vp, vp, vp, vp, vp]
    return L


def _ptr(a):
    return None if a is None else a.ctypes.data


# --------------------------------------------------------------------------- primitives
def philox(key, ctr):
    """Philox-4x32-10 of one (key[2], ctr[4]) -> 4 uint32."""
    k = np.ascontiguousarray(key, dtype=np.uint32)
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_ptr(k), _ptr(c), _ptr(o))
    return o


def exp(x: float) -> float:
    return lib().orc_exp(float(x))


def threshold(h: float, beta: float) -> int:
    return int(lib().orc_threshold(float(h), float(beta)))


def field(Jc: float, s: int, q: float, sigma: int, lam: float) -> float:
    return lib().orc_field(float(Jc), int(s), float(q), int(sigma), float(lam))


def draw_plane(seed, a, b, t, half, k) -> int:
    return int(lib().orc_draw_plane(seed, a, b, t, half, k))


def draw_direct(seed, a, b, t, half, k) -> int:
    return int(lib().orc_draw_direct(seed, a, b, t, half, k))


# --------------------------------------------------------------------------- lattice
def _frozen(frozen, n):
    if frozen is None:
        return None
    f = np.ascontiguousarray(frozen, dtype=np.uint8).reshape(-1)
    assert f.size == n
    return f


def lattice_init(L, R, seed, mode=MODE_SINGLE, kind=0, frozen=None):
    s = np.zeros((R, L, L), dtype=np.int8)
    f = _frozen(frozen, L * L)
    lib().orc_lattice_init(_ptr(s), L, R, _ptr(f), seed, mode, kind)
    return s


def lattice_half(s, J, q, lam, beta, seed, t, half, mode=MODE_SINGLE, frozen=None):
    s = np.ascontiguousarray(s, dtype=np.int8)
    R, L, _ = s.shape
    out = np.empty_like(s)
    b = np.ascontiguousarray(np.broadcast_to(np.asarray(beta, dtype=np.float64), (R,)))
    f = _frozen(frozen, L * L)
    lib().orc_lattice_half(_ptr(s), _ptr(out), L, R, _ptr(f), J, q, lam, _ptr(b), seed, t, half,
                           mode)
    return out


def lattice_site(s_r, i, j, J, q, lam, beta, seed, t, half, mode, r, frozen=None):
    """tau at site (i, j) of replica r given that replica's configuration s_r [L][L]."""
    s_r = np.ascontiguousarray(s_r, dtype=np.int8)
    L = s_r.shape[0]
    f = _frozen(frozen, L * L)
    return lib().orc_lattice_site(_ptr(s_r), L, i, j, _ptr(f), J, q, lam, beta, seed, t, half,
                                  mode, r)


def lattice_run(s, J, q, lam, beta, seed, t0, n_steps, mode=MODE_SINGLE, frozen=None):
    """n_steps full steps from s (R, L, L); returns (sigma, sigma')."""
    s = np.array(s, dtype=np.int8, order="C", copy=True)
    R, L, _ = s.shape
    sp = s.copy()
    b = np.ascontiguousarray(np.broadcast_to(np.asarray(beta, dtype=np.float64), (R,)))
    f = _frozen(frozen, L * L)
    lib().orc_lattice_run(_ptr(s), _ptr(sp), L, R, _ptr(f), J, q, lam, _ptr(b), seed, t0,
                          n_steps, mode)
    return s, sp


def lattice_anneal(s, J, q, lam, beta_sched, seed, t0, mode=MODE_SINGLE, frozen=None):
    s = np.array(s, dtype=np.int8, order="C", copy=True)
    R, L, _ = s.shape
    sp = s.copy()
    b = np.ascontiguousarray(beta_sched, dtype=np.float64)
    f = _frozen(frozen, L * L)
    lib().orc_lattice_anneal(_ptr(s), _ptr(sp), L, R, _ptr(f), J, q, lam, _ptr(b), seed, t0,
                             b.size, mode)
    return s, sp


def lattice_sums(s_r, sp_r):
    """Integer sums (M, E, P1, P2, M2, cut) of one replica."""
    a = np.ascontiguousarray(s_r, dtype=np.int8)
    b = np.ascontiguousarray(sp_r, dtype=np.int8)
    out = np.zeros(6, dtype=np.int64)
    lib().orc_lattice_sums(_ptr(a), _ptr(b), a.shape[0], _ptr(out))
    return out


def lattice_observables(s, sp, J, q, lam):
    """Per replica: dict of m, H (Eq. ham1 with field 2 lambda), pair energy, cut."""
    R, L, _ = s.shape
    res = []
    for r in range(R):
        M, E, P1, P2, M2, cut = (int(v) for v in lattice_sums(s[r], sp[r]))
        H = -(J * E) - 2.0 * lam * M
        Hp = -(J * P1 + q * P2 + lam * (M + M2))
        res.append(dict(M=M, E=E, P1=P1, P2=P2, M2=M2, m=M / (L * L), H=H, pair=Hp, cut=cut))
    return res


# --------------------------------------------------------------------------- graphs
def orient(u, v, rule=0):
    u = np.ascontiguousarray(u, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    tail = np.empty_like(u)
    head = np.empty_like(v)
    lib().orc_orient(u.size, _ptr(u), _ptr(v), rule, _ptr(tail), _ptr(head))
    return tail, head


def graph_init(n, R, seed, kind=0, frozen=None):
    s = np.zeros((R, n), dtype=np.int8)
    f = _frozen(frozen, n)
    lib().orc_graph_init(_ptr(s), n, R, _ptr(f), seed, kind)
    return s


def graph_half(s, tail, head, J, integer_J, lam, q, beta, seed, t, half, frozen=None,
               draw=DRAW_DIRECT):
    s = np.ascontiguousarray(s, dtype=np.int8)
    R, n = s.shape
    out = np.empty_like(s)
    tail = np.ascontiguousarray(tail, dtype=np.int32)
    head = np.ascontiguousarray(head, dtype=np.int32)
    Jd = np.ascontiguousarray(J, dtype=np.float64)
    ld = np.ascontiguousarray(np.broadcast_to(np.asarray(lam, dtype=np.float64), (n,)))
    b = np.ascontiguousarray(np.broadcast_to(np.asarray(beta, dtype=np.float64), (R,)))
    f = _frozen(frozen, n)
    lib().orc_graph_half(_ptr(s), _ptr(out), n, tail.size, _ptr(tail), _ptr(head), _ptr(Jd),
                         int(integer_J), _ptr(f), _ptr(ld), q, _ptr(b), R, seed, t, half,
                         int(draw))
    return out


def graph_fields(s, tail, head, J, integer_J, lam, q, half):
    """Fields h[R][n] (fp64) of one half step on the configurations s [R][n]."""
    s = np.ascontiguousarray(s, dtype=np.int8)
    R, n = s.shape
    h = np.empty((R, n), dtype=np.float64)
    tail = np.ascontiguousarray(tail, dtype=np.int32)
    head = np.ascontiguousarray(head, dtype=np.int32)
    Jd = np.ascontiguousarray(J, dtype=np.float64)
    ld = np.ascontiguousarray(np.broadcast_to(np.asarray(lam, dtype=np.float64), (n,)))
    lib().orc_graph_fields(_ptr(s), _ptr(h), n, tail.size, _ptr(tail), _ptr(head), _ptr(Jd),
                           int(integer_J), _ptr(ld), q, R, half)
    return h


class Incidence:
    """Incidence lists of one half step (orc_incidence) with the per-vertex oracle
    routines that use them: the field, the draw and the decision of one (x, r)."""

    def __init__(self, n, tail, head, J, integer_J, lam, q, half, frozen=None):
        self.n, self.half, self.q, self.integer_J = n, half, float(q), int(integer_J)
        self.tail = np.ascontiguousarray(tail, dtype=np.int32)
        self.head = np.ascontiguousarray(head, dtype=np.int32)
        self.J = np.ascontiguousarray(J, dtype=np.float64)
        self.lam = np.ascontiguousarray(np.broadcast_to(np.asarray(lam, dtype=np.float64), (n,)))
        self.frozen = _frozen(frozen, n)
        self.start = np.zeros(n + 1, dtype=np.int64)
        self.list = np.zeros(max(self.tail.size, 1), dtype=np.int64)
        lib().orc_incidence(n, self.tail.size, _ptr(self.tail), _ptr(self.head), half,
                            _ptr(self.start), _ptr(self.list))

    def field(self, sr, x):
        sr = np.ascontiguousarray(sr, dtype=np.int8)
        return lib().orc_graph_field(_ptr(sr), int(x), _ptr(self.start), _ptr(self.list),
                                     _ptr(self.tail), _ptr(self.head), _ptr(self.J),
                                     self.integer_J, _ptr(self.lam), self.q, self.half)

    def site(self, sr, x, r, beta, seed, t, draw=DRAW_DIRECT):
        sr = np.ascontiguousarray(sr, dtype=np.int8)
        return lib().orc_graph_site(_ptr(sr), int(x), _ptr(self.start), _ptr(self.list),
                                    _ptr(self.tail), _ptr(self.head), _ptr(self.J),
                                    self.integer_J, _ptr(self.frozen), _ptr(self.lam), self.q,
                                    float(beta), seed, t, self.half, int(draw), int(r))


def graph_draw(seed, x, r, t, half, draw) -> int:
    return int(lib().orc_graph_draw(seed, int(x), int(r), t, half, int(draw)))


def graph_draws(seed, n, R, t, half, draw):
    """u[R][n]: the draw of every (replica, vertex) of one half step."""
    u = np.empty((R, n), dtype=np.uint32)
    lib().orc_graph_draws(_ptr(u), n, R, seed, t, half, int(draw))
    return u


def graph_run(s, tail, head, J, integer_J, lam, q, beta, seed, t0, n_steps, beta_sched=None,
              frozen=None, draw=DRAW_DIRECT):
    s = np.array(s, dtype=np.int8, order="C", copy=True)
    R, n = s.shape
    sp = s.copy()
    tail = np.ascontiguousarray(tail, dtype=np.int32)
    head = np.ascontiguousarray(head, dtype=np.int32)
    Jd = np.ascontiguousarray(J, dtype=np.float64)
    ld = np.ascontiguousarray(np.broadcast_to(np.asarray(lam, dtype=np.float64), (n,)))
    b = np.ascontiguousarray(np.broadcast_to(np.asarray(beta, dtype=np.float64), (R,)))
    bs = None if beta_sched is None else np.ascontiguousarray(beta_sched, dtype=np.float64)
    if bs is not None:
        n_steps = bs.size
    f = _frozen(frozen, n)
    lib().orc_graph_run(_ptr(s), _ptr(sp), n, tail.size, _ptr(tail), _ptr(head), _ptr(Jd),
                        int(integer_J), _ptr(f), _ptr(ld), q, _ptr(b), _ptr(bs), R, seed, t0,
                        n_steps, int(draw))
    return s, sp


def graph_sums(s_r, sp_r, tail, head, J, lam):
    a = np.ascontiguousarray(s_r, dtype=np.int8)
    b = np.ascontiguousarray(sp_r, dtype=np.int8)
    tail = np.ascontiguousarray(tail, dtype=np.int32)
    head = np.ascontiguousarray(head, dtype=np.int32)
    Jd = np.ascontiguousarray(J, dtype=np.float64)
    ld = np.ascontiguousarray(np.broadcast_to(np.asarray(lam, dtype=np.float64), (a.size,)))
    out = np.zeros(7, dtype=np.float64)
    lib().orc_graph_sums(_ptr(a), _ptr(b), a.size, tail.size, _ptr(tail), _ptr(head), _ptr(Jd),
                         _ptr(ld), _ptr(out))
    return out


def graph_observables(s, sp, tail, head, J, lam, q):
    R, n = s.shape
    res = []
    for r in range(R):
        S, E, Lm, P1, P2, L2, cut = graph_sums(s[r], sp[r], tail, head, J, lam)
        H = -E - 2.0 * Lm
        Hp = -(P1 + q * P2 + Lm + L2)
        res.append(dict(M=S, E=E, LS=Lm, m=S / n, H=H, pair=Hp, cut=cut))
    return res
