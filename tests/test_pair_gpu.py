"""The SM-pair form of the fused tensor-core RowSel kernel (tile variant 7:
clusters of 2 CTAs, cta_group::2 MMAs with M = 256 sharing one database tile)
against the CPU oracle, bit-exact.

Shapes are chosen for the pair's own bookkeeping: an even number of 32-row
m-blocks (the odd CTA's block ragged or full), ragged k and n, more than 8
exact 512-row groups per unit (a Barrett flush mid-unit), a digit ring that
wraps, rings smaller than 8 slots, and the fallback to the single-CTA form
when the batch has an odd number of m-blocks."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TC = 4
PAIR_VARIANT = 7


@pytest.fixture(scope="module")
def g():
    from tests import gpu_util
    lib = gpu_util.lib()
    if lib.gpir_num_variants(TC) <= PAIR_VARIANT:
        pytest.skip("tensor-core path without the pair variant")
    return lib


def _run(g, ct, db, B, N, primes, trace=False):
    from tests.gpu_util import DbHandle, to_dev, to_host
    h = DbHandle(g, db, N, primes, path_mask=TC)
    try:
        g.gpir_set_variant(h.h, B, TC, PAIR_VARIANT)
        if trace:
            g.gpir_trace_enable(True)
            g.gpir_trace_read()
        try:
            got = to_host(h.rowsel(to_dev(ct), B, TC))
            names = [n for n, _ in g.gpir_trace_read()] if trace else []
        finally:
            if trace:
                g.gpir_trace_enable(False)
    finally:
        h.close()
    return got, names


SHAPES = [
    # (B, D0, D1, L, N, primes)                      what it covers
    (17, 70, 40, 2, 64, synth.PRIMES_28),           # 2 m-blocks, the odd CTA's ragged (M = 34); ragged k, n
    (32, 300, 70, 2, 128, synth.PRIMES_28),         # 2 full m-blocks, 2 n-blocks (second ragged)
    (64, 600, 130, 2, 32, synth.PRIMES_28),         # 4 m-blocks, 3 n-blocks, two 512-row groups
    (20, 4500, 8, 1, 16, synth.PRIMES_28[:1]),      # 9 groups: a Barrett flush after 8, then the last
    (18, 130, 70, 2, 512, synth.PRIMES_28),         # 256 ring entries: the digit ring wraps
    (32, 40, 24, 2, 4, (17, 41)),                   # N = 4: 4 valid slots of an 8-slot group
    (9, 70, 40, 2, 64, synth.PRIMES_28),            # 1 m-block: the single-CTA form runs instead
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "B%d_D0%d_D1%d_L%d_N%d" % s[:5])
def test_pair_vs_oracle(g, shape):
    from tests.gpu_util import make_problem
    B, D0, D1, L, N, primes = shape
    ct, db = make_problem(2000 + B + D0, B, D0, D1, L, N, primes)
    got, _ = _run(g, ct, db, B, N, primes)
    want = oracle.rowsel(ct, db, list(primes))
    assert np.array_equal(got, want), "%d of %d differ" % (int((got != want).sum()), want.size)


def test_pair_kernel_is_the_one_that_runs(g):
    """With an even number of m-blocks the launch is the pair kernel; with an
    odd number, the single-CTA fused kernel."""
    from tests.gpu_util import make_problem
    primes = synth.PRIMES_28
    for B, name in ((17, "tc_pair"), (9, "tc_fused")):
        ct, db = make_problem(2100 + B, B, 70, 40, 2, 64, primes)
        got, names = _run(g, ct, db, B, 64, primes, trace=True)
        assert name in names and ("tc_pair" in names) == (name == "tc_pair"), names
        assert np.array_equal(got, oracle.rowsel(ct, db, list(primes)))


@pytest.mark.parametrize("a,b", [(None, None), (0x7F7F80, 0x7F7F80), (0x7F7F7F, 0x7F7F7F)])
def test_pair_extreme_accumulation(g, a, b):
    """All residues q - 1 (result D0 mod q), and the residues whose balanced
    digits all sit at the ends of their range (result D0 a b mod q), over
    D0 = 2048 rows with two m-blocks."""
    primes = synth.PRIMES_28
    B, D0, D1, L, N = 17, 2048, 8, 2, 32
    ct = np.empty((B, D0, 2, L, N), dtype=np.uint32)
    db = np.empty((D0, D1, L, N), dtype=np.uint32)
    for l, q in enumerate(primes):
        ct[:, :, :, l] = q - 1 if a is None else a
        db[:, :, l] = q - 1 if b is None else b
    got, _ = _run(g, ct, db, B, N, primes)
    for l, q in enumerate(primes):
        want = D0 % q if a is None else (D0 * a * b) % q
        assert np.all(got[:, :, :, l] == want)


@pytest.mark.parametrize("name,n_slots", [("c2_rowsel", 6), ("c4_large", 4)])
def test_pair_full_size_sampled(g, name, n_slots):
    """The 32-client and the 4 GiB workloads through the pair kernel; oracle on
    sampled slots."""
    from tests.test_parity_gpu import _sampled_full_size
    _sampled_full_size(g, name, TC, n_slots=n_slots, variant=PAIR_VARIANT)
