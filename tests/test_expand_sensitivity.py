"""Plant plausible mistakes in a copy of the ExpandQuery oracle (on the CPU) and
check that at least one ExpandQuery pin rejects each."""

import numpy as np
import pytest

import oracle
import synth
from tests import expand_util as eu

PRIMES = synth.PRIMES_28


def _auto_coeffs(a, k, q, v):
    a = [int(x) for x in a]
    N = len(a)
    out = [0] * N
    for i, ai in enumerate(a):
        e = (i * k) % (2 * N)
        if e < N or v == "no_sign":
            out[e % N] = (out[e % N] + ai) % q
        else:
            out[e - N] = (out[e - N] - ai) % q
    return np.array(out, dtype=np.uint64)


def _auto_ntt(A, k, q, v):
    N = len(A)
    psi = oracle.psi_2n(q, N)
    return oracle.ntt_negacyclic(_auto_coeffs(oracle.intt_negacyclic(A, q, psi), k, q, v), q, psi)


def _subs(ct, k, evk, primes, v):
    L = len(primes)
    ct = np.asarray(ct)
    N = ct.shape[-1]
    ell = oracle.gadget_digits(primes)
    ta = np.stack([_auto_ntt(ct[0][l], k, q, v) for l, q in enumerate(primes)])
    tb = np.stack([(ct[1][l].astype(np.uint64) if v == "no_tau_b" else _auto_ntt(ct[1][l], k, q, v))
                   for l, q in enumerate(primes)])
    digits = oracle.decompose(ct[0] if v == "dcp_before_tau" else ta, primes, ell)
    out = np.zeros((2, L, N), dtype=np.uint64)
    out[1] = tb
    for i in range(ell):
        for l, q in enumerate(primes):
            d = oracle.ntt_negacyclic([di % q for di in digits[i]], q, oracle.psi_2n(q, N))
            for r in range(2):
                rr = 1 - r if v == "evk_swap" else r
                out[r, l] = (out[r, l] + (d * np.asarray(evk[i][rr][l], dtype=np.uint64)) % np.uint64(q)) % np.uint64(q)
    return out.astype(np.uint32)


def _node(ct, j, evk_j, primes, v):
    ct = np.asarray(ct)
    N = ct.shape[-1]
    k = N // (1 << j) - 1 if v == "k_minus" else N // (1 << j) + 1
    t = _subs(ct, k, evk_j, primes, v).astype(np.int64)
    c = ct.astype(np.int64)
    qv = np.array(primes, dtype=np.int64).reshape(1, -1, 1)
    out0 = ((c + t) % qv).astype(np.uint64)
    diff = ((c + t) % qv if v == "out1_sum" else (c - t) % qv).astype(np.uint64)
    e = (1 << j) if v == "x_plus" else -(1 << j)
    out1 = np.stack([np.stack([(diff[r, l] * oracle.monomial_ntt(e, q, N)) % np.uint64(q)
                               for l, q in enumerate(primes)]) for r in range(2)])
    return out0.astype(np.uint32), out1.astype(np.uint32)


def _expand(query, evk, primes, v):
    level = [np.asarray(query)]
    for j in range(len(evk)):
        outs = [_node(c, j, evk[j], primes, v) for c in level]
        if v == "interleaved":
            level = [x for pair in outs for x in pair]
        else:
            level = [o[0] for o in outs] + [o[1] for o in outs]
    return level


def pin_subs_phase(v):
    N = 16
    ell = oracle.gadget_digits(PRIMES)
    query, _, s, m = eu.toy_expand_inputs(5, 0, 2, N, PRIMES, ell)
    for k in (N + 1, 9):
        evk = eu.toy_evk(5, 0, k, s, 2, N, PRIMES, ell)
        got = eu.phase_coeffs(_subs(query, k, evk, PRIMES, v), s, PRIMES)
        for l, q in enumerate(PRIMES):
            assert got[l] == [int(x) for x in oracle.automorphism_coeffs([x % q for x in m], k, q)]


def pin_tree(v):
    N, J = 16, 3
    ell = oracle.gadget_digits(PRIMES)
    query, evk, s, m = eu.toy_expand_inputs(12, J, 2, N, PRIMES, ell)
    out = _expand(query, evk, PRIMES, v)
    for r in range(1 << J):
        assert eu.phase_coeffs(out[r], s, PRIMES) == eu.expected_output_coeffs(m, J, r, N, PRIMES)


PINS = [pin_subs_phase, pin_tree]
MUTANTS = ["no_sign", "no_tau_b", "dcp_before_tau", "evk_swap", "k_minus", "out1_sum", "x_plus", "interleaved"]


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
    assert caught, "no ExpandQuery pin caught mutant %s" % variant
