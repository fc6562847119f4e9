"""The device-side failure path on the GPU: a bounded wait that runs out (an
mbarrier that nothing arrives on, waited through the helper the RowSel kernels
use) is reported by gpir_sync as GPIR_ETIMEOUT, the following sync is clean,
and the context stays usable: RowSel afterwards is still bit-exact. No trap, no
fault, no unbounded wait."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_expired_device_wait_is_reported_and_the_context_survives():
    from tests import gpu_util
    from tests.gpu_util import DbHandle, to_dev, to_host, make_problem
    g = gpu_util.lib()
    assert g.gpir_sync_rc(None, 20000) == g.GPIR_OK            # nothing pending, no stale error
    g.gpir_selftest_bounded_wait(None)
    assert g.gpir_sync_rc(None, 20000) == g.GPIR_ETIMEOUT      # the wait gave up after its 2 s limit
    assert g.gpir_sync_rc(None, 20000) == g.GPIR_OK            # reading the error word cleared it
    primes = synth.PRIMES_28
    B, D0, D1, L, N = 3, 40, 24, 2, 64
    ct, db = make_problem(71, B, D0, D1, L, N, primes)
    want = oracle.rowsel(ct, db, list(primes))
    h = DbHandle(g, db, N, primes, path_mask=0)
    try:
        for path in (1, 4):
            if g.gpir_num_variants(path):
                assert np.array_equal(to_host(h.rowsel(to_dev(ct), B, path)), want), path
    finally:
        h.close()


def test_injected_allocation_failures_leave_handles_usable():
    """Host-side allocation-failure injection (gpir_set_fail_alloc): the
    database upload, the growth of a tensor-core workspace on a new stream and
    the host-buffer entry point's workspace each return GPIR_ENOMEM when their
    allocation is made to fail, and the same calls then succeed bit-exactly
    with the injection disarmed. No GPU memory is exhausted."""
    import torch
    from tests import gpu_util
    from tests.gpu_util import to_dev, to_host, make_problem
    g = gpu_util.lib()
    primes = synth.PRIMES_28
    B, D0, D1, L, N = 3, 40, 24, 2, 64
    ct, db = make_problem(72, B, D0, D1, L, N, primes)
    want = oracle.rowsel(ct, db, list(primes))
    params = g.gpir_params_create(N, list(primes))
    h = None
    try:
        g.gpir_set_fail_alloc(1)
        with pytest.raises(g.GpirError) as ei:
            g.gpir_db_upload(params, D0, D1, to_dev(db), True, 0)
        assert ei.value.code == g.GPIR_ENOMEM
        # second allocation of the upload (the tensor-core digit tiles)
        g.gpir_set_fail_alloc(2)
        with pytest.raises(g.GpirError) as ei:
            g.gpir_db_upload(params, D0, D1, to_dev(db), True, 0)
        assert ei.value.code == g.GPIR_ENOMEM
        assert g.gpir_set_fail_alloc(0) == 0
        h = g.gpir_db_upload(params, D0, D1, to_dev(db), True, 0)
        # workspace growth on a stream that has none yet
        st = torch.cuda.Stream()
        ct_d = to_dev(ct)
        out = torch.full((B, D1, 2, L, N), -1, dtype=torch.int32, device="cuda")
        g.gpir_set_fail_alloc(1)
        with pytest.raises(g.GpirError) as ei:
            g.gpir_rowsel_batch(h, B, ct_d, out, g.GPIR_PATH_TC, st)
        assert ei.value.code == g.GPIR_ENOMEM
        g.gpir_set_fail_alloc(0)
        g.gpir_rowsel_batch(h, B, ct_d, out, g.GPIR_PATH_TC, st)
        st.synchronize()
        assert np.array_equal(to_host(out), want)
        # host-buffer entry point: its ciphertext workspace
        out_h = np.zeros((B, D1, 2, L, N), dtype=np.uint32)
        g.gpir_set_fail_alloc(1)
        with pytest.raises(g.GpirError) as ei:
            g.gpir_rowsel_batch_host(h, B, np.ascontiguousarray(ct), out_h, 1)
        assert ei.value.code == g.GPIR_ENOMEM
        g.gpir_set_fail_alloc(0)
        g.gpir_rowsel_batch_host(h, B, np.ascontiguousarray(ct), out_h, 1)
        g.gpir_sync(None, 20000)
        assert np.array_equal(out_h, want)
    finally:
        g.gpir_set_fail_alloc(0)
        if h is not None:
            g.gpir_db_free(h)
        g.gpir_params_destroy(params)
