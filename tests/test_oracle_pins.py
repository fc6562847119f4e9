"""The CPU oracle pinned to facts outside itself (runs without a GPU)."""

import numpy as np
import pytest

import oracle
import synth
from tests import pins


# ---- primes and roots (Sec. 2.4.1: NTT-friendly RNS primes) -----------------

def test_primes_below_2_28():
    p = oracle.ntt_friendly_primes(4096, 28, 4)
    assert p[:2] == list(synth.PRIMES_28) == [268369921, 268361729]
    for q in p:
        assert oracle.is_prime(q) and q < 2 ** 28 and (q - 1) % 8192 == 0
    # nothing prime and NTT-friendly between the two and 2^28
    for q in range(p[0] + 8192, 2 ** 28, 8192):
        assert not oracle.is_prime(q)
    assert oracle.ntt_friendly_primes(2048, 28, 2) == [268369921, 268361729]


@pytest.mark.parametrize("q,n", [(17, 4), (41, 4), (97, 8), (193, 16), (257, 32), (268369921, 2048),
                                 (268361729, 4096)])
def test_psi_is_primitive_2n_root(q, n):
    psi = oracle.psi_2n(q, n)
    assert pow(psi, n, q) == q - 1          # psi^n = -1
    assert pow(psi, 2 * n, q) == 1


def test_is_prime_small_table():
    primes = [x for x in range(2, 200) if oracle.is_prime(x)]
    assert primes[:10] == [2, 3, 5, 7, 11, 13, 17, 19, 23, 29] and len(primes) == 46


# ---- negacyclic NTT vs schoolbook multiplication -----------------------------

@pytest.mark.parametrize("q,n", [(17, 4), (41, 4), (17, 8), (97, 8), (97, 16), (193, 16), (193, 32), (257, 32)])
def test_ntt_convolution_tiny(q, n):
    rng = np.random.default_rng(q * n)
    psi = oracle.psi_2n(q, n)
    for _ in range(3):
        a = rng.integers(0, q, n)
        b = rng.integers(0, q, n)
        A = oracle.ntt_negacyclic(a, q, psi)
        Bv = oracle.ntt_negacyclic(b, q, psi)
        assert np.array_equal(oracle.intt_negacyclic(A, q, psi), a.astype(np.uint64))
        c = oracle.schoolbook_negacyclic(a, b, q)
        assert np.array_equal(oracle.ntt_negacyclic(c, q, psi), (A * Bv) % np.uint64(q))


def test_schoolbook_textbook_case():
    # X * X^(n-1) = X^n = -1 in Z_q[X]/(X^n + 1)
    q, n = 97, 8
    x = np.zeros(n, dtype=np.int64); x[1] = 1
    y = np.zeros(n, dtype=np.int64); y[n - 1] = 1
    c = oracle.schoolbook_negacyclic(x, y, q)
    assert c[0] == q - 1 and not c[1:].any()


def test_ntt_of_one_is_all_ones():
    q, n = 268369921, 64
    psi = oracle.psi_2n(q, n)
    e = np.zeros(n, dtype=np.uint64); e[0] = 1
    assert np.all(oracle.ntt_negacyclic(e, q, psi) == 1)


def test_ntt_convolution_n2048():
    q, n = synth.PRIMES_28[0], 2048
    psi = oracle.psi_2n(q, n)
    rng = np.random.default_rng(2048)
    a = rng.integers(0, q, n)
    b = np.zeros(n, dtype=np.int64)
    b[rng.integers(0, n, 6)] = rng.integers(0, q, 6)   # sparse b keeps the Python schoolbook fast
    c = oracle.schoolbook_negacyclic(a, b, q)
    A = oracle.ntt_negacyclic(a, q, psi)
    Bv = oracle.ntt_negacyclic(b, q, psi)
    assert np.array_equal(oracle.ntt_negacyclic(c, q, psi), (A * Bv) % np.uint64(q))
    assert np.array_equal(oracle.intt_negacyclic(A, q, psi), a.astype(np.uint64))


# ---- RowSel pins ---------------------------------------------------------------

@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_rowsel_pins(pin):
    pin(oracle.rowsel)


def test_rowsel_output_matches_rowsel():
    primes = synth.PRIMES_28
    ct = synth.ct_tensor(9, 3, 11, 2, 16, primes)
    db = synth.db_tensor(9, 11, 5, 2, 16, primes)
    out = oracle.rowsel(ct, db, list(primes))
    rng = np.random.default_rng(0)
    for _ in range(40):
        c, j, r, l, t = (int(rng.integers(0, s)) for s in (3, 5, 2, 2, 16))
        assert oracle.rowsel_output(ct, db, primes, c, j, r, l, t) == int(out[c, j, r, l, t])


def test_rowsel_slot_subset_independence():
    """Slot-wise independence: RowSel on a slot subset equals the subset of RowSel."""
    primes = synth.PRIMES_28
    ct = synth.ct_tensor(11, 2, 9, 2, 32, primes)
    db = synth.db_tensor(11, 9, 4, 2, 32, primes)
    full = oracle.rowsel(ct, db, list(primes))
    sel = np.array([0, 5, 31, 17])
    part = oracle.rowsel(ct[..., sel], db[..., sel], list(primes))
    assert np.array_equal(part, full[..., sel])


def test_rowsel_large_d0_no_overflow():
    """D0 = 5000 rows of (q-1)*(q-1): the uint64 sum of reduced products stays exact."""
    primes = synth.PRIMES_28
    D0 = 5000
    ct = np.empty((1, D0, 2, 2, 4), dtype=np.uint32)
    db = np.empty((D0, 1, 2, 4), dtype=np.uint32)
    for l, q in enumerate(primes):
        ct[:, :, :, l] = q - 1
        db[:, :, l] = q - 1
    out = oracle.rowsel(ct, db, list(primes))
    for l, q in enumerate(primes):
        assert np.all(out[:, :, :, l] == D0 % q)
