"""Plant plausible mistakes in a copy of the ColTor oracle (on the CPU) and check
that at least one ColTor pin rejects each."""

import numpy as np
import pytest

import oracle
import synth

PRIMES = synth.PRIMES_28
Z = 1 << oracle.GADGET_LOG_BASE


def _decompose(poly_ntt, primes, ell, v):
    N = len(poly_ntt[0])
    if v == "no_intt":
        coef = [np.asarray(poly_ntt[l], dtype=np.uint64) for l in range(len(primes))]
    else:
        coef = [oracle.intt_negacyclic(poly_ntt[l], q, oracle.psi_2n(q, N)) for l, q in enumerate(primes)]
    xs = oracle.crt_centered(coef, primes)
    if v == "no_center":
        Q = int(np.prod([int(q) for q in primes], dtype=object))
        xs = [x % Q for x in xs]
    z = (1 << 23) if v == "base23" else Z
    digits = [[0] * N for _ in range(ell)]
    for j, x in enumerate(xs):
        for i, di in enumerate(oracle.balanced_digits(x, z, ell)):
            digits[i][j] = di
    return digits


def _external_product(rgsw, ct, primes, v):
    L = len(primes)
    ct = np.asarray(ct)
    N = ct.shape[-1]
    ell = oracle.gadget_digits(primes)
    use = ell - 1 if v == "drop_last_digit" else ell
    out = np.zeros((2, L, N), dtype=np.uint64)
    for p in range(2):
        digits = _decompose(ct[p], primes, ell, v)
        for i in range(use):
            row_idx = i * 2 + p if v == "row_order" else p * ell + i
            for l, q in enumerate(primes):
                d = oracle.ntt_negacyclic([di % q for di in digits[i]], q, oracle.psi_2n(q, N))
                for r in range(2):
                    row = np.asarray(rgsw[row_idx][r][l], dtype=np.uint64)
                    out[r, l] = (out[r, l] + (d * row) % np.uint64(q)) % np.uint64(q)
    return out.astype(np.uint32)


def _coltor(ct, rgsw, primes, v):
    qv = np.array(primes, dtype=np.int64).reshape(1, -1, 1)
    level = [np.asarray(c) for c in ct]
    stages = len(rgsw)
    s = 0
    while len(level) > 1:
        nxt = []
        for k in range(len(level) // 2):
            lo = level[2 * k].astype(np.int64)
            hi = level[2 * k + 1].astype(np.int64)
            if v == "cmux_swap":
                lo, hi = hi, lo
            st = stages - 1 - s if v == "bit_order_msb" else s
            ep = _external_product(rgsw[st], ((hi - lo) % qv).astype(np.uint32), primes, v).astype(np.int64)
            nxt.append((ep % qv if v == "cmux_no_lo" else (lo + ep) % qv).astype(np.uint32))
        level = nxt
        s += 1
    return level[0]


def _phase(ct, s, primes):
    return [[(int(b) - int(a) * int(si)) % q for a, b, si in zip(ct[0][l], ct[1][l], s[l])]
            for l, q in enumerate(primes)]


def pin_external_product_decrypts(v):
    N, L = 16, 2
    ell = oracle.gadget_digits(PRIMES)
    s = synth.uniform_residues(11, synth.TAG_SECRET, (L, N), PRIMES, limb_axis=0)
    a = synth.uniform_residues(12, synth.TAG_MASK, (L, N), PRIMES, limb_axis=0).astype(np.int64)
    mu = synth.uniform_residues(13, synth.TAG_RECORD, (L, N), PRIMES, limb_axis=0).astype(np.int64)
    qv = np.array(PRIMES, dtype=np.int64)[:, None]
    ct = np.stack([a, (a * s.astype(np.int64) + mu) % qv]).astype(np.uint32)
    for m in (0, 1, 3):
        rgsw = synth.toy_rgsw(11, 0, m, s, L, N, PRIMES, ell)
        out = _external_product(rgsw, ct, PRIMES, v)
        assert _phase(out, s, PRIMES) == [[(m * int(x)) % q for x in mu[l]] for l, q in enumerate(PRIMES)]


def pin_tournament(v):
    N, L, D1 = 8, 2, 8
    ell = oracle.gadget_digits(PRIMES)
    for jstar in range(D1):
        ct, rgsw, s, rec = synth.toy_coltor_inputs(31 + jstar, D1, L, N, PRIMES, jstar, ell)
        out = _coltor(ct, rgsw, PRIMES, v)
        assert _phase(out, s, PRIMES) == [[int(x) for x in rec[jstar][l]] for l in range(L)]


def pin_digit_ranges(v):
    N = 32
    Q = PRIMES[0] * PRIMES[1]
    rng = np.random.default_rng(3)
    coeffs = [int(x) for x in rng.integers(-(Q // 2) + 1, Q // 2, N)]
    poly_ntt = [oracle.ntt_negacyclic([c % q for c in coeffs], q, oracle.psi_2n(q, N)) for q in PRIMES]
    digits = _decompose(poly_ntt, PRIMES, 3, v)
    for j in range(N):
        assert sum(digits[i][j] * Z ** i for i in range(3)) == coeffs[j]
        assert all(-(Z // 2) <= digits[i][j] < Z // 2 for i in range(2))
        assert abs(digits[2][j]) <= Q // (2 * Z * Z) + 1


PINS = [pin_external_product_decrypts, pin_tournament, pin_digit_ranges]
MUTANTS = ["row_order", "base23", "no_center", "no_intt", "drop_last_digit", "cmux_no_lo", "cmux_swap",
           "bit_order_msb"]


def test_unmutated_copy_passes_all_pins():
    for pin in PINS:
        pin("none")


@pytest.mark.parametrize("variant", MUTANTS)
def test_mutant_is_caught(variant):
    caught = []
    for pin in PINS:
        try:
            pin(variant)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, "no ColTor pin caught mutant %s" % variant
