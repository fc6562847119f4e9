"""The allocation-free RowSel entry point (gpir_rowsel_batch_noalloc).

Callers that cannot allocate device memory while they run -- code under a
CUDA stream capture, or services whose device memory is fixed at start-up --
use this entry point; it keeps the tensor-core path's digit-tile workspace in
a fixed array inside the library. These tests call it through the C ABI and
check that it returns exactly what the oracle and the regular entry point
return, on two calls in a row (the shared array keeps the previous call's
contents, which must not leak into the next result). This file is named so pytest collects it
last.
"""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from tests import gpu_util
    return gpu_util.lib()


def test_noalloc_matches_regular_entry_point_twice(g):
    """Two calls in a row on the shared array: first a larger problem (two
    32-row m-blocks, three 64-row k-chunks), then a smaller one whose m-rows
    and k-rows are both padded inside their tiles, so leftovers of the first
    call sit where the second reads padding. Each output must equal the
    oracle's and the regular entry point's, bit for bit."""
    import torch
    import oracle
    from tests.gpu_util import DbHandle, to_dev, to_host
    if g.gpir_num_variants(g.GPIR_PATH_TC) == 0:
        pytest.skip("tensor-core path not built")
    primes = synth.PRIMES_28
    L, N = 2, 256
    # (B, D0, D1): 512 slots x 2 m-blocks x 3 k-chunks x 16 KiB = 48 MiB, then
    # 512 slots x 1 m-block x 2 k-chunks x 16 KiB = 16 MiB
    for call, (B, D0, D1, seed) in enumerate(((20, 130, 40, 22), (5, 70, 24, 23))):
        ct_np = synth.ct_tensor(seed, B, D0, L, N, primes)
        db_np = synth.db_tensor(seed, D0, D1, L, N, primes)
        want = oracle.rowsel(ct_np, db_np, list(primes))
        h = DbHandle(g, db_np, N, primes, path_mask=g.GPIR_PATH_TC)
        try:
            ct = to_dev(ct_np)
            ref = torch.full((B, D1, 2, L, N), -1, dtype=torch.int32, device="cuda")
            g.gpir_rowsel_batch(h.h, B, ct, ref, g.GPIR_PATH_TC)
            out = torch.full((B, D1, 2, L, N), -7, dtype=torch.int32, device="cuda")
            g.gpir_rowsel_batch_noalloc(h.h, B, ct, out)
            torch.cuda.synchronize()
            g.gpir_sync(None, 20000)
            a, b = to_host(out), to_host(ref)
            assert np.array_equal(a, want), "call %d: %d of %d outputs differ from the oracle" % (
                call, int((a != want).sum()), a.size)
            assert np.array_equal(a, b), "call %d: %d of %d outputs differ from gpir_rowsel_batch" % (
                call, int((a != b).sum()), a.size)
        finally:
            h.close()


def test_noalloc_rejects_oversized_problem(g):
    import torch
    from tests.gpu_util import DbHandle, to_dev
    if g.gpir_num_variants(g.GPIR_PATH_TC) == 0:
        pytest.skip("tensor-core path not built")
    primes = synth.PRIMES_28
    B, D0, D1, L, N = 20, 64, 8, 2, 4096       # 8192 slots x 2 m-blocks x 1 k-chunk x 16 KiB = 256 MiB
    db = synth.db_tensor(24, D0, D1, L, N, primes)
    h = DbHandle(g, db, N, primes, path_mask=g.GPIR_PATH_TC)
    try:
        ct = torch.zeros(B * D0 * 2 * L * N, dtype=torch.int32, device="cuda")
        out = torch.zeros(B * D1 * 2 * L * N, dtype=torch.int32, device="cuda")
        with pytest.raises(g.GpirError) as ei:
            g.gpir_rowsel_batch_noalloc(h.h, B, ct, out)
        assert ei.value.code == g.GPIR_ETOOBIG
    finally:
        h.close()
