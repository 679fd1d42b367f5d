"""Philox-4x32-10 from an independent implementation (Triton's ``tl.philox``),
executed on the CPU by the Triton interpreter.  Used only as a test reference.

Usage: python triton_philox_ref.py  < json {"seed": s, "ctrs": [[c0,c1,c2,c3], ...]}
prints json [[o0,o1,o2,o3], ...].
"""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _kern(out, c0p, c1p, c2p, c3p, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c0p + i)
    c1 = tl.load(c1p + i)
    c2 = tl.load(c2p + i)
    c3 = tl.load(c3p + i)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out + i * 4 + 0, a)
    tl.store(out + i * 4 + 1, b)
    tl.store(out + i * 4 + 2, c)
    tl.store(out + i * 4 + 3, d)


def main():
    req = json.load(sys.stdin)
    ctrs = np.asarray(req["ctrs"], dtype=np.uint64).astype(np.uint32)
    n = ctrs.shape[0]
    N = 1
    while N < n:
        N *= 2
    pad = np.zeros((N, 4), dtype=np.uint32)
    pad[:n] = ctrs
    out = torch.zeros(4 * N, dtype=torch.int32)
    cols = [torch.from_numpy(pad[:, k].view(np.int32).copy()) for k in range(4)]
    _kern[(1,)](out, *cols, int(req["seed"]), N=N)
    res = out.numpy().view(np.uint32).reshape(N, 4)[:n]
    json.dump(res.astype(np.int64).tolist(), sys.stdout)


if __name__ == "__main__":
    main()
