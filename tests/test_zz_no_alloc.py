"""The allocation-free observables entry point (shaken_lattice_observables_noalloc).

It serves callers that cannot call cudaMalloc (all their device memory comes
from their own pool or caching allocator, or they cannot afford the
synchronisation an allocation may imply): its reduction scratch is a fixed
device array inside the library.  Checked through the C ABI against the
regular entry point (shaken_observables) on the same state, twice in a row so
that stale scratch from the first call would show.  This file is collected
last; it passes alone in a fresh process and after the other tests."""
import numpy as np
import pytest

from tests.gpu_util import lattice_problem, lib, require_cuda

pytestmark = pytest.mark.gpu

HEADER_BYTES = 56  # checkpoint header: magic, version, kind, enc, R, n, step, bytes, flags


def device_state(S, ctx):
    import torch
    ck = S.shaken_save(ctx)
    nb = int.from_bytes(ck[40:48], "little")
    a = np.frombuffer(ck, dtype=np.uint8, count=nb, offset=HEADER_BYTES).copy()
    b = np.frombuffer(ck, dtype=np.uint8, count=nb, offset=HEADER_BYTES + nb).copy()
    return torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()


@pytest.mark.parametrize("enc,L,R,J,q,lam", [
    ("INT8", 96, 3, 1.0, 0.5, 0.01),
    ("PACKED", 64, 2, -0.7, 1.0, -0.2),
    ("MULTISPIN", 64, 64, 1.0, 1.0, 0.0),
    # the grid's x dimension at its cap of 1024 blocks: a grid-stride loop, and
    # several blocks adding into the same replica's sums
    ("INT8", 4096, 1, 1.0, 1.0, 0.0),
    # the scratch's replica limit exactly (128 multispin groups)
    ("MULTISPIN", 32, 4096, 1.0, 0.8, 0.05),
])
def test_noalloc_observables_match_regular_entry(enc, L, R, J, q, lam):
    require_cuda()
    S = lib()
    e = getattr(S, enc)
    beta = np.linspace(0.3, 0.6, R)
    ctx = S.shaken_init(lattice_problem(S, e, L, R, beta, J, q, lam), 2024 + L)
    try:
        for call in range(2):
            S.shaken_step(ctx, 3 + 4 * call)
            A, B = device_state(S, ctx)
            ref = S.shaken_observables(ctx, R)
            got = S.shaken_lattice_observables_noalloc(A.data_ptr(), B.data_ptr(), e, L, R, J, q,
                                                       lam)
            for f in ("magnetization", "energy", "pair_energy", "cut_weight"):
                assert np.allclose(got[f], ref[f], rtol=0, atol=1e-9), (call, f)
            assert np.array_equal(got["cut_edges"], ref["cut_edges"])
    finally:
        S.shaken_free(ctx)


def test_noalloc_rejects_too_many_replicas():
    require_cuda()
    S = lib()
    import torch
    buf = torch.zeros(64 * 64 * 4097, dtype=torch.uint8, device="cuda")
    with pytest.raises(S.ShakenError) as ei:
        S.shaken_lattice_observables_noalloc(buf.data_ptr(), buf.data_ptr(), S.INT8, 64, 4097,
                                             1.0, 1.0, 0.0)
    assert ei.value.status == -1 and "4096" in str(ei.value)
