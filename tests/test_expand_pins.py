"""Pins of the ExpandQuery oracle (GPIR paper Sec. 2.2 "ExpandQuery", Sec. 2.5.1).

Each test checks the oracle against something other than itself: the
automorphism against direct evaluation of the polynomial at the roots of
X^N + 1 and against the NTT-domain slot permutation, monomial products against
the schoolbook product, Subs against the decryption identity under noiseless
toy keys and against a coefficient-domain schoolbook key switch, and the whole
tree against the coefficient split it is built to perform.
"""

import numpy as np
import pytest

import oracle
import synth
from tests import expand_util as eu

PRIMES = synth.PRIMES_28
SMALL = (97, 193)          # N = 16: q = 1 mod 32


def _eval(coeffs, x, q):
    acc = 0
    for c in reversed(list(coeffs)):
        acc = (acc * x + int(c)) % q
    return acc


@pytest.mark.parametrize("k", [3, 5, 9, 17, 31])
def test_automorphism_is_substitution_at_the_roots(k):
    """tau_k(a) evaluated at zeta = psi^(2s+1) equals a evaluated at zeta^k."""
    q, N = 97, 16
    psi = oracle.psi_2n(q, N)
    rng = np.random.default_rng(k)
    a = rng.integers(0, q, N)
    t = oracle.automorphism_coeffs(a, k, q)
    for s in range(N):
        z = pow(psi, 2 * s + 1, q)
        assert _eval(t, z, q) == _eval(a, pow(z, k, q), q)


def test_automorphism_group_laws():
    q, N = 193, 16
    rng = np.random.default_rng(1)
    a = rng.integers(0, q, N)
    assert np.array_equal(oracle.automorphism_coeffs(a, 1, q), a.astype(np.uint64))
    for k1, k2 in [(3, 5), (17, 9), (31, 31), (N + 1, N + 1)]:
        lhs = oracle.automorphism_coeffs(oracle.automorphism_coeffs(a, k1, q), k2, q)
        assert np.array_equal(lhs, oracle.automorphism_coeffs(a, (k1 * k2) % (2 * N), q))
    # tau_{2N-1}: X -> X^-1 = -X^(N-1)
    t = oracle.automorphism_coeffs(a, 2 * N - 1, q)
    assert int(t[0]) == int(a[0]) and all(int(t[N - i]) == (-int(a[i])) % q for i in range(1, N))


@pytest.mark.parametrize("N,q", [(16, 97), (64, PRIMES[0]), (256, PRIMES[1])])
def test_automorphism_ntt_is_slot_permutation(N, q):
    rng = np.random.default_rng(N)
    A = rng.integers(0, q, N).astype(np.uint64)
    for j in range(3):
        k = N // (1 << j) + 1
        assert np.array_equal(oracle.automorphism_ntt(A, k, q), A[eu.slot_perm(N, k)])


def test_monomial_ntt_against_schoolbook():
    q, N = 193, 16
    psi = oracle.psi_2n(q, N)
    rng = np.random.default_rng(2)
    p = rng.integers(0, q, N)
    P = oracle.ntt_negacyclic(p, q, psi)
    for e in [1, 2, 5, 15, -1, -4, -16, 16, 31]:
        x = [0] * N
        ee = e % (2 * N)
        x[ee % N] = 1 if ee < N else q - 1
        want = oracle.ntt_negacyclic(oracle.schoolbook_negacyclic(x, p, q), q, psi)
        assert np.array_equal((oracle.monomial_ntt(e, q, N) * P) % np.uint64(q), want)
    for e in [1, 3, 8]:
        prod = (oracle.monomial_ntt(e, q, N) * oracle.monomial_ntt(-e, q, N)) % np.uint64(q)
        assert np.all(prod == 1)


@pytest.mark.parametrize("L", [1, 2])
def test_subs_decrypts_to_substituted_phase(L):
    """Noiseless toy keys: phase(Subs(ct, k)) = tau_k(phase(ct)) exactly."""
    primes = PRIMES[:L]
    N = 16
    ell = oracle.gadget_digits(primes)
    query, _, s, m = eu.toy_expand_inputs(5, 0, L, N, primes, ell)
    for k in [N + 1, N // 2 + 1, 3, 2 * N - 1]:
        evk = eu.toy_evk(5, 0, k, s, L, N, primes, ell)
        out = oracle.subs(query, k, evk, primes)
        got = eu.phase_coeffs(out, s, primes)
        for l, q in enumerate(primes):
            assert got[l] == [int(x) for x in oracle.automorphism_coeffs([x % q for x in m], k, q)]


def test_subs_key_switch_matches_coefficient_domain_schoolbook():
    """The NTT-domain multiply-accumulate equals the same sum with negacyclic
    schoolbook products on coefficients, plus tau_k(b)."""
    primes = PRIMES
    N, k = 16, 9
    ell = oracle.gadget_digits(primes)
    rng = np.random.default_rng(7)
    evk = np.stack([np.stack([np.stack([rng.integers(0, q, N) for q in primes]) for _ in range(2)])
                    for _ in range(ell)]).astype(np.uint32)
    ct = np.stack([np.stack([rng.integers(0, q, N) for q in primes]) for _ in range(2)]).astype(np.uint32)
    got = oracle.subs(ct, k, evk, primes)
    ta = np.stack([ct[0][l][eu.slot_perm(N, k)] for l in range(2)])
    digits = oracle.decompose(ta, primes, ell)
    for l, q in enumerate(primes):
        psi = oracle.psi_2n(q, N)
        for r in range(2):
            acc = [0] * N
            for i in range(ell):
                row = oracle.intt_negacyclic(evk[i][r][l], q, psi)
                prod = oracle.schoolbook_negacyclic([d % q for d in digits[i]], row, q)
                acc = [(x + int(y)) % q for x, y in zip(acc, prod)]
            want = oracle.ntt_negacyclic(acc, q, psi)
            if r == 1:
                want = (want + ct[1][l][eu.slot_perm(N, k)].astype(np.uint64)) % np.uint64(q)
            assert np.array_equal(got[r][l].astype(np.uint64), want)


@pytest.mark.parametrize("j", [0, 1, 3])
def test_node_outputs_split_even_and_odd(j):
    """Stage j node: phase(out0) = M + tau(M), phase(out1) = X^(-2^j) (M - tau(M))."""
    primes = PRIMES
    N = 16
    ell = oracle.gadget_digits(primes)
    query, _, s, m = eu.toy_expand_inputs(9, 0, 2, N, primes, ell)
    k = N // (1 << j) + 1
    evk = eu.toy_evk(9, j, k, s, 2, N, primes, ell)
    o0, o1 = oracle.expand_node(query, j, evk, primes)
    p0, p1 = eu.phase_coeffs(o0, s, primes), eu.phase_coeffs(o1, s, primes)
    for l, q in enumerate(primes):
        mq = [x % q for x in m]
        tm = [int(x) for x in oracle.automorphism_coeffs(mq, k, q)]
        assert p0[l] == [(a + b) % q for a, b in zip(mq, tm)]
        diff = [(a - b) % q for a, b in zip(mq, tm)]
        xinv = [0] * N
        e = (-(1 << j)) % (2 * N)
        xinv[e % N] = 1 if e < N else q - 1
        assert p1[l] == [int(x) for x in oracle.schoolbook_negacyclic(xinv, diff, q)]


@pytest.mark.parametrize("L,N,J", [(1, 16, 4), (2, 16, 4), (2, 16, 2), (2, 32, 3)])
def test_tree_splits_message_into_coefficients(L, N, J):
    """Output r after J stages decrypts to 2^J sum_i m_{2^J i + r} X^(2^J i)."""
    primes = PRIMES[:L]
    ell = oracle.gadget_digits(primes)
    query, evk, s, m = eu.toy_expand_inputs(11 + J, J, L, N, primes, ell)
    out = oracle.expand_query(query, evk, primes, 1 << J)
    assert out.shape == (1 << J, 2, L, N)
    for r in range(1 << J):
        assert eu.phase_coeffs(out[r], s, primes) == eu.expected_output_coeffs(m, J, r, N, primes), r


def test_one_hot_query_selects_row():
    """A query whose message is X^(i*) expands (J = log2 N) into ciphertexts of
    N [r = i*]: the one-hot selection vector RowSel consumes, up to the known
    factor N."""
    primes = PRIMES
    N, J = 16, 4
    ell = oracle.gadget_digits(primes)
    istar = 11
    query, evk, s, _ = eu.toy_expand_inputs(21, J, 2, N, primes, ell)
    # re-encrypt the message X^istar under the same key
    for l, q in enumerate(primes):
        M = oracle.monomial_ntt(istar, q, N)
        a = query[0, l].astype(np.uint64)
        query[1, l] = ((a * s[l].astype(np.uint64) + M) % np.uint64(q)).astype(np.uint32)
    out = oracle.expand_query(query, evk, primes, N)
    for r in range(N):
        for l, q in enumerate(primes):
            want = [N % q if (r == istar and i == 0) else 0 for i in range(N)]
            assert eu.phase_coeffs(out[r], s, primes)[l] == want


def test_n_out_is_a_prefix():
    primes = PRIMES
    N, J = 16, 3
    ell = oracle.gadget_digits(primes)
    query, evk, s, m = eu.toy_expand_inputs(31, J, 2, N, primes, ell)
    full = oracle.expand_query(query, evk, primes, 8)
    for n_out in (1, 5, 8):
        assert np.array_equal(oracle.expand_query(query, evk, primes, n_out), full[:n_out])
    with pytest.raises(ValueError):
        oracle.expand_query(query, evk, primes, 9)


@pytest.mark.parametrize("istar,jstar", [(0, 0), (5, 3), (7, 1)])
def test_three_phases_return_the_scaled_record(istar, jstar):
    """ExpandQuery of a query encrypting X^(i*) gives the one-hot selection
    vector (scaled by 2^J), RowSel selects row i*, ColTor with RGSW bits of j*
    selects column j*: the result decrypts to 2^J DB[i*][j*] (noiseless toy
    keys, N = 16)."""
    primes = PRIMES
    N, L, D0, D1, J = 16, 2, 8, 4, 3
    ell = oracle.gadget_digits(primes)
    db = synth.uniform_residues(51, synth.TAG_DB, (D0, D1, L, N), primes, limb_axis=2)
    query, evk, s, _ = eu.toy_expand_inputs(52, J, L, N, primes, ell)
    for l, q in enumerate(primes):
        M = oracle.monomial_ntt(istar, q, N)
        query[1, l] = ((query[0, l].astype(np.uint64) * s[l].astype(np.uint64) + M) % np.uint64(q)).astype(np.uint32)
    sel = oracle.expand_query(query, evk, primes, D0)                    # [D0][2][L][N]
    rows = oracle.rowsel(sel[None], db, primes)[0]                        # [D1][2][L][N]
    rgsw = np.stack([synth.toy_rgsw(53, st, (jstar >> st) & 1, s, L, N, primes, ell) for st in range(2)])
    out = oracle.coltor(rows, rgsw, primes)
    for l, q in enumerate(primes):
        ph = [(int(bb) - int(aa) * int(ss)) % q for aa, bb, ss in zip(out[0][l], out[1][l], s[l])]
        assert ph == [((1 << J) * int(x)) % q for x in db[istar][jstar][l]]
