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
