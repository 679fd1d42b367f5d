"""Shared helpers of the GPU parity tests: build/load the CUDA library and run
problems through the C ABI."""
import numpy as np
import pytest


def lib():
    """The CUDA binding; builds libshaken.so if needed.  Fails (does not skip)
    when the library cannot be built or loaded."""
    from paper_1904_06257_gb300 import build
    build.build()
    from paper_1904_06257_gb300 import shaken as S
    return S


def require_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")


def lattice_problem(S, enc, L, R, beta, J=1.0, q=1.0, lam=0.0, frozen=None, init=0,
                    init_spins=None):
    return S.Problem(S.LATTICE, enc, R, beta, q, L=L, J=J, lambda_const=lam,
                     boundary=0, frozen_mask=frozen, init=init, init_spins=init_spins)


def graph_problem(S, n, u, v, J, R, beta, q=1.0, lam=None, lam_c=0.0, integer=True,
                  orientation=0, frozen=None, init=0, init_spins=None):
    return S.Problem(S.GRAPH, S.MULTISPIN, R, beta, q, n=n, u=u, v=v, J_edge=J,
                     J_is_integer=integer, orientation=orientation, lambda_=lam,
                     lambda_const=lam_c, frozen_mask=frozen, init=init, init_spins=init_spins)


def graph_spins_from_raw(raw, n, R):
    """int8 [R][n] spins from a graph's raw MULTISPIN state (uint32 [n][R/32], bit k of the
    word of vertex x in group g = replica 32 g + k; the layout of shaken_get_state_raw)."""
    words = np.frombuffer(np.ascontiguousarray(raw).tobytes(), dtype=np.uint32)
    words = words.reshape(n, R // 32).T
    bits = (words[:, None, :] >> np.arange(32, dtype=np.uint32)[None, :, None]) & 1
    return np.where(bits.reshape(R, n) != 0, 1, -1).astype(np.int8)
