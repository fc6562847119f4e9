"""Pin checks for a RowSel implementation with the oracle's signature.

Each check raises AssertionError when the implementation disagrees with what
the GPIR paper and the mathematics fix. They are applied to the oracle in
test_oracle_pins.py, and to deliberately broken copies of it (planted on the
CPU) in test_pin_sensitivity.py to show each plausible mistake is caught.
"""

import numpy as np

import oracle
import synth

TINY = {8: (17, 97), 16: (97, 193), 32: (193, 257)}


def _ring_polys(rng, shape, primes, limb_axis):
    out = np.empty(shape, dtype=np.uint32)
    idx = [slice(None)] * len(shape)
    for l, q in enumerate(primes):
        idx[limb_axis] = l
        sub = out[tuple(idx)]
        out[tuple(idx)] = rng.integers(0, q, size=sub.shape, dtype=np.uint64).astype(np.uint32)
    return out


def check_ring_semantics(rowsel, n=8, B=2, D0=3, D1=2, seed=0):
    """Sec. 2.4.1: NTT(a*b) = NTT(a) (.) NTT(b). So INTT of each RowSel output
    must equal sum_i ct_i * DB[i][j] computed as negacyclic polynomials."""
    primes = TINY[n]
    rng = np.random.default_rng(seed)
    L = len(primes)
    ct = _ring_polys(rng, (B, D0, 2, L, n), primes, 3)
    db = _ring_polys(rng, (D0, D1, L, n), primes, 2)
    out = rowsel(ct, db, list(primes))
    for l, q in enumerate(primes):
        psi = oracle.psi_2n(q, n)
        for c in range(B):
            for r in range(2):
                for j in range(D1):
                    want = np.zeros(n, dtype=np.int64)
                    for i in range(D0):
                        a = oracle.intt_negacyclic(ct[c, i, r, l], q, psi)
                        b = oracle.intt_negacyclic(db[i, j, l], q, psi)
                        want = (want + oracle.schoolbook_negacyclic(a, b, q).astype(np.int64)) % q
                    got = oracle.intt_negacyclic(out[c, j, r, l], q, psi)
                    assert np.array_equal(got.astype(np.int64), want), (l, c, r, j)


def check_one_hot(rowsel, N=16, D0=5, D1=3, seed=1):
    """Sec. 2.2: the selection cts encrypt 0 except the i*-th, which encrypts 1.
    With plaintext 'ciphertexts' (e, e) where e = NTT(1) = all ones, RowSel must
    return DB row i* exactly, for each client's own i*."""
    primes = synth.PRIMES_28
    L = 2
    istars = [4, 0, 2]
    B = len(istars)
    db = synth.db_tensor(seed, D0, D1, L, N, primes)
    ct = np.zeros((B, D0, 2, L, N), dtype=np.uint32)
    for c, i in enumerate(istars):
        ct[c, i] = 1
    out = rowsel(ct, db, list(primes))
    for c, i in enumerate(istars):
        for r in range(2):
            assert np.array_equal(out[c, :, r], db[i]), (c, r)


def check_toy_rlwe(rowsel, N=32, D0=6, D1=4, seed=2):
    """Noiseless toy RLWE in the NTT domain: ct_i = (a_i, a_i s + [i = i*]).
    RowSel is linear, so out_b - out_a (.) s must equal DB[i*][j] exactly."""
    primes = synth.PRIMES_28
    L = 2
    db = synth.db_tensor(seed, D0, D1, L, N, primes)
    istars = [3, 5]
    cts, secrets = [], []
    for c, i in enumerate(istars):
        ct, s = synth.toy_rlwe_selection(seed * 10 + c, D0, L, N, primes, i)
        cts.append(ct)
        secrets.append(s)
    ct = np.stack(cts)
    out = rowsel(ct, db, list(primes))
    for c, i in enumerate(istars):
        for l, q in enumerate(primes):
            for j in range(D1):
                got = oracle.rlwe_decrypt_ntt(out[c, j, 0, l], out[c, j, 1, l], secrets[c][l], q)
                assert np.array_equal(got, db[i, j, l]), (c, l, j)


def check_linearity(rowsel, N=8, B=2, D0=7, D1=3, seed=3):
    """RowSel(alpha ct + beta ct') = alpha RowSel(ct) + beta RowSel(ct') mod q,
    and the same in the database argument."""
    primes = synth.PRIMES_28
    L = 2
    rng = np.random.default_rng(seed)
    ct1 = synth.ct_tensor(seed, B, D0, L, N, primes)
    ct2 = synth.ct_tensor(seed + 100, B, D0, L, N, primes)
    db1 = synth.db_tensor(seed, D0, D1, L, N, primes)
    db2 = synth.db_tensor(seed + 100, D0, D1, L, N, primes)
    alpha, beta = [int(x) for x in rng.integers(1, 1 << 27, size=2)]

    def comb(x, y, limb_axis):
        z = np.empty_like(x)
        for l, q in enumerate(primes):
            idx = [slice(None)] * x.ndim
            idx[limb_axis] = l
            xi = x[tuple(idx)].astype(object)
            yi = y[tuple(idx)].astype(object)
            z[tuple(idx)] = ((alpha * xi + beta * yi) % q).astype(np.uint32)
        return z

    lhs = rowsel(comb(ct1, ct2, 3), db1, list(primes))
    rhs = comb(rowsel(ct1, db1, list(primes)), rowsel(ct2, db1, list(primes)), 3)
    assert np.array_equal(lhs, rhs)
    lhs = rowsel(ct1, comb(db1, db2, 2), list(primes))
    rhs = comb(rowsel(ct1, db1, list(primes)), rowsel(ct1, db2, list(primes)), 3)
    assert np.array_equal(lhs, rhs)


def check_closed_forms(rowsel, N=8, B=2, D0=300, D1=3, seed=4):
    """All residues q-1: (q-1)^2 = 1 mod q, so every output is D0 mod q (per
    limb, with distinct primes). All-ones ct: column sums of the DB mod q.
    Zero ct: zero."""
    primes = synth.PRIMES_28
    L = 2
    ct = np.empty((B, D0, 2, L, N), dtype=np.uint32)
    db = np.empty((D0, D1, L, N), dtype=np.uint32)
    for l, q in enumerate(primes):
        ct[:, :, :, l] = q - 1
        db[:, :, l] = q - 1
    out = rowsel(ct, db, list(primes))
    for l, q in enumerate(primes):
        assert np.all(out[:, :, :, l] == D0 % q)
    db = synth.db_tensor(seed, D0, D1, L, N, primes)
    ones = np.ones((B, D0, 2, L, N), dtype=np.uint32)
    out = rowsel(ones, db, list(primes))
    for l, q in enumerate(primes):
        colsum = (db[:, :, l].astype(np.uint64).sum(axis=0) % np.uint64(q)).astype(np.uint32)  # [D1][N]
        for c in range(B):
            for r in range(2):
                assert np.array_equal(out[c, :, r, l], colsum)
    zero = np.zeros_like(ones)
    assert not rowsel(zero, db, list(primes)).any()


def check_brute_force(rowsel, N=4, B=2, D0=3, D1=2, seed=5):
    """Tiny shapes: every output against a Python big-integer sum."""
    primes = (17, 41)
    ct = synth.ct_tensor(seed, B, D0, 2, N, primes)
    db = synth.db_tensor(seed, D0, D1, 2, N, primes)
    out = rowsel(ct, db, list(primes))
    for c in range(B):
        for j in range(D1):
            for r in range(2):
                for l, q in enumerate(primes):
                    for t in range(N):
                        s = sum(int(ct[c, i, r, l, t]) * int(db[i, j, l, t]) for i in range(D0))
                        assert int(out[c, j, r, l, t]) == s % q


ALL_PINS = [check_ring_semantics, check_one_hot, check_toy_rlwe, check_linearity, check_closed_forms,
            check_brute_force]
