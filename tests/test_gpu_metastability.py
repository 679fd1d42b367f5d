"""The metastable regime of Sec. 3.2 on the GPU (0 < q < lambda < J, large beta):
from the all-minus configuration the chain leaves -1 at a rate fixed, to first order,
by the single-site flip probability 1 / (1 + e^{2 beta (2J + q - lambda)}) of the
proof of Thm 3.3 (tests.test_oracle_pins.exit_probability_per_step), so the mean
exit time grows like e^{2 beta (2J + q - lambda)} (the time scale of Thm 3.1).
Multispin lattices, 512 replicas of a 32 x 32 torus, m recorded every full step."""
import math

import numpy as np
import pytest

from tests.gpu_util import lattice_problem, lib, require_cuda
from tests.test_oracle_pins import exit_probability_per_step, exit_rate_mle

pytestmark = pytest.mark.gpu

J, Q, LAM = 1.0, 0.1, 0.15  # the parameters of the paper's metastability runs


@pytest.fixture(scope="module")
def S():
    require_cuda()
    return lib()


def first_exits(S, L, beta, groups, steps, seed):
    """Step (1-based) of each replica's first full-step configuration other than -1
    (0: none within `steps`), and whether it reached +1 by the end."""
    first, plus = [], []
    for g in range(groups):
        ctx = S.shaken_init(lattice_problem(S, S.MULTISPIN, L, 32, beta, J, Q, LAM, init=2),
                            seed + g)
        mag, _ = S.shaken_step_record(ctx, steps, 32)
        S.shaken_free(ctx)
        out = mag > -1.0
        f = np.where(out.any(axis=0), out.argmax(axis=0) + 1, 0)
        first.append(f)
        plus.append((mag == 1.0).any(axis=0))
    return np.concatenate(first), np.concatenate(plus)


@pytest.mark.parametrize("beta,steps", [(3.0, 400), (3.5, 2500), (4.0, 8000)])
def test_exit_rate_from_minus(S, beta, steps):
    L = 32
    first, _ = first_exits(S, L, beta, 16, steps, 0x5348414B + int(10 * beta))
    P = exit_probability_per_step(J, Q, LAM, beta, L * L)
    Phat, exits = exit_rate_mle(first, steps)
    assert exits > 100
    assert abs(Phat - P) < 4 * Phat / math.sqrt(exits), (beta, Phat, P, exits)
