"""Slot-sharded RowSel through the library (paper Sec. 6, database sharding):
every shard of a W-way split runs on this one GPU in turn (each a complete,
independent RowSel on a ring of N / W points; no shard waits on another), and
the reassembled output equals the oracle's, bit for bit."""

import numpy as np
import pytest

import oracle
import synth
from paper_2604_04696_gb300 import shard

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from tests import gpu_util
    return gpu_util.lib()


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("path,variant", [(4, 0), (4, 8), (1, None)])
def test_shards_reassemble_to_the_oracle(g, world, path, variant):
    from tests.gpu_util import DbHandle, to_dev, to_host
    if g.gpir_num_variants(path) == 0:
        pytest.skip("path not built")
    primes = synth.PRIMES_28
    B, D0, D1, L, N = 5, 70, 40, 2, 256
    ct = synth.ct_tensor(81, B, D0, L, N, primes)
    db = synth.db_tensor(81, D0, D1, L, N, primes)
    parts = []
    for r in range(world):
        sh = shard.SlotShard(N, world, r)
        h = DbHandle(g, sh.take(db), sh.T, primes, path_mask=path)
        try:
            if variant is not None:
                g.gpir_set_variant(h.h, B, path, variant)
            parts.append(to_host(h.rowsel(to_dev(sh.take(ct)), B, path)))
        finally:
            h.close()
    assert np.array_equal(shard.assemble(parts), oracle.rowsel(ct, db, list(primes)))
