"""Pins of the ColTor oracle (GPIR paper Sec. 2.2 "ColTor", Sec. 2.5.1).

Each test checks the oracle against something other than itself: the CRT and
digit identities, the decryption identity of an external product under
noiseless toy encryptions, a coefficient-domain schoolbook recomputation of the
external product, and the whole tournament decrypting to the chosen record.
"""

import numpy as np
import pytest

import oracle
import synth

PRIMES = synth.PRIMES_28


def _phase(ct, s, primes):
    """b - a (.) s mod q, per limb (noiseless toy decryption, NTT domain)."""
    out = []
    for l, q in enumerate(primes):
        a = np.asarray(ct[0][l], dtype=object)
        b = np.asarray(ct[1][l], dtype=object)
        out.append([(int(bi) - int(ai) * int(si)) % q for ai, bi, si in zip(a, b, s[l])])
    return out


def test_gadget_digit_count():
    # z = 2^22: Q < 2^28 needs 2 digits, Q < 2^56 needs 3 (the paper: 5 digits for Q ~ 2^108)
    assert oracle.gadget_digits(PRIMES[:1]) == 2
    assert oracle.gadget_digits(PRIMES) == 3
    assert oracle.gadget_digits([2 ** 27 + 1] * 4) == 5


def test_crt_centered_reconstructs_residues():
    rng = np.random.default_rng(1)
    res = [rng.integers(0, q, 64) for q in PRIMES]
    xs = oracle.crt_centered(res, PRIMES)
    Q = PRIMES[0] * PRIMES[1]
    for j, x in enumerate(xs):
        assert -Q // 2 < x <= Q // 2
        for l, q in enumerate(PRIMES):
            assert x % q == int(res[l][j])
    # the extremes of the centred range
    assert oracle.crt_centered([[0], [0]], PRIMES) == [0]
    assert oracle.crt_centered([[q - 1] for q in PRIMES], PRIMES) == [-1]


def test_balanced_digits_reconstruct_within_range():
    z = 1 << oracle.GADGET_LOG_BASE
    Q = PRIMES[0] * PRIMES[1]
    rng = np.random.default_rng(2)
    xs = [int(v) for v in rng.integers(-(Q // 2) + 1, Q // 2, 500)] + [Q // 2, -(Q // 2) + 1, 0, -1, 1,
                                                                      z // 2, -(z // 2), z // 2 - 1]
    for x in xs:
        d = oracle.balanced_digits(x, z, 3)
        assert sum(di * z ** i for i, di in enumerate(d)) == x
        assert all(-(z // 2) <= di < z // 2 for di in d[:-1])
        assert abs(d[-1]) <= Q // (2 * z * z) + 1     # centring keeps the top digit small


def test_decompose_recovers_centred_coefficients():
    N = 32
    rng = np.random.default_rng(3)
    Q = PRIMES[0] * PRIMES[1]
    coeffs = [int(v) for v in rng.integers(-(Q // 2) + 1, Q // 2, N)]
    poly_ntt = [oracle.ntt_negacyclic([c % q for c in coeffs], q, oracle.psi_2n(q, N)) for q in PRIMES]
    digits = oracle.decompose(poly_ntt, PRIMES, 3)
    z = 1 << oracle.GADGET_LOG_BASE
    for j in range(N):
        assert sum(digits[i][j] * z ** i for i in range(3)) == coeffs[j]


@pytest.mark.parametrize("L", [1, 2])
@pytest.mark.parametrize("m", [0, 1, 3])
def test_external_product_decrypts_to_m_times_phase(L, m):
    primes = PRIMES[:L]
    N = 16
    ell = oracle.gadget_digits(primes)
    s = synth.uniform_residues(11, synth.TAG_SECRET, (L, N), primes, limb_axis=0)
    rgsw = synth.toy_rgsw(11, 0, m, s, L, N, primes, ell)
    a = synth.uniform_residues(12, synth.TAG_MASK, (L, N), primes, limb_axis=0).astype(np.int64)
    mu = synth.uniform_residues(13, synth.TAG_RECORD, (L, N), primes, limb_axis=0).astype(np.int64)
    qv = np.array(primes, dtype=np.int64)[:, None]
    ct = np.stack([a, (a * s.astype(np.int64) + mu) % qv]).astype(np.uint32)
    out = oracle.external_product(rgsw, ct, primes)
    ph = _phase(out, s, primes)
    for l, q in enumerate(primes):
        assert ph[l] == [(m * int(v)) % q for v in mu[l]]


def test_external_product_matches_coefficient_domain_schoolbook():
    """The NTT-domain multiply-accumulate equals the same sum computed with
    negacyclic schoolbook products on coefficients (then transformed)."""
    primes = PRIMES
    N = 16
    ell = oracle.gadget_digits(primes)
    rng = np.random.default_rng(5)
    rgsw = np.stack([np.stack([np.stack([rng.integers(0, q, N) for q in primes]) for _ in range(2)])
                     for _ in range(2 * ell)]).astype(np.uint32)
    ct = np.stack([np.stack([rng.integers(0, q, N) for q in primes]) for _ in range(2)]).astype(np.uint32)
    got = oracle.external_product(rgsw, ct, primes)
    for l, q in enumerate(primes):
        psi = oracle.psi_2n(q, N)
        for r in range(2):
            acc = [0] * N
            for p in range(2):
                digits = oracle.decompose(ct[p], primes, ell)
                for i in range(ell):
                    row = oracle.intt_negacyclic(rgsw[p * ell + i][r][l], q, psi)
                    prod = oracle.schoolbook_negacyclic([d % q for d in digits[i]], row, q)
                    acc = [(x + int(y)) % q for x, y in zip(acc, prod)]
            want = oracle.ntt_negacyclic(acc, q, psi)
            assert np.array_equal(got[r][l].astype(np.uint64), want)


@pytest.mark.parametrize("L", [1, 2])
def test_cmux_selects_by_bit(L):
    primes = PRIMES[:L]
    N = 8
    ell = oracle.gadget_digits(primes)
    ct, rgsw, s, rec = synth.toy_coltor_inputs(21, 2, L, N, primes, 1, ell)
    out1 = oracle.cmux(rgsw[0], ct[0], ct[1], primes)
    assert _phase(out1, s, primes) == [[int(v) for v in rec[1][l]] for l in range(L)]
    ct, rgsw, s, rec = synth.toy_coltor_inputs(21, 2, L, N, primes, 0, ell)
    out0 = oracle.cmux(rgsw[0], ct[0], ct[1], primes)
    assert _phase(out0, s, primes) == [[int(v) for v in rec[0][l]] for l in range(L)]


@pytest.mark.parametrize("L", [1, 2])
def test_tournament_decrypts_to_selected_record(L):
    primes = PRIMES[:L]
    N, D1 = 16, 8
    ell = oracle.gadget_digits(primes)
    for jstar in range(D1):
        ct, rgsw, s, rec = synth.toy_coltor_inputs(31 + jstar, D1, L, N, primes, jstar, ell)
        out = oracle.coltor(ct, rgsw, primes)
        assert _phase(out, s, primes) == [[int(v) for v in rec[jstar][l]] for l in range(L)]


def test_rowsel_then_coltor_returns_db_entry():
    """RowSel with a toy one-hot query, then ColTor over its D1 outputs, decrypts
    to DB[i*][j*] (noiseless toy encryptions, small ring)."""
    primes = PRIMES
    N, L, D0, D1 = 8, 2, 4, 4
    ell = oracle.gadget_digits(primes)
    db = synth.uniform_residues(41, synth.TAG_DB, (D0, D1, L, N), primes, limb_axis=2)
    istar, jstar = 2, 3
    ct, s = synth.toy_rlwe_selection(41, D0, L, N, primes, istar)
    rows = oracle.rowsel(ct[None], db, primes)[0]                       # [D1][2][L][N]
    rgsw = np.stack([synth.toy_rgsw(41, st, (jstar >> st) & 1, s, L, N, primes, ell) for st in range(2)])
    out = oracle.coltor(rows, rgsw, primes)
    assert _phase(out, s, primes) == [[int(v) for v in db[istar][jstar][l]] for l in range(L)]
