"""ExpandQuery by its definition (test infrastructure; see the package docstring).

GPIR paper, Sec. 2.2 ("ExpandQuery") and Sec. 2.5.1 (the steps of Subs). The
server turns one query ciphertext into 2^J ciphertexts with a binary tree of J
stages; every tree node takes one ciphertext and returns two, through one
homomorphic substitution (Subs) with the stage's evaluation key (evk).

Subs(ct, k, evk), ct = (a, b) in the NTT domain:
  1. the automorphism tau_k: X -> X^k applied to a and to b
     (coefficient i of a polynomial moves to i k mod 2N, negated when that
     lands at or above N, since X^N = -1);
  2. key switching, with Dcp on tau_k(a) only (Sec. 2.5.1): inverse NTT, CRT
     reconstruction centred to (-Q/2, Q/2], balanced base-2^22 digits
     d_0..d_{ell-1}, forward NTT of each digit polynomial, then
         a' = sum_i NTT(d_i) (.) evk[i][0]
         b' = tau_k(b) + sum_i NTT(d_i) (.) evk[i][1].

Tree node at stage j (0-based) on ciphertext c, with k_j = N / 2^j + 1:
    t    = Subs(c, k_j, evk_j)
    out0 = c + t
    out1 = X^(-2^j) (c - t)
Stage j maps the list [c_0 .. c_{2^j - 1}] to a list twice as long, with
out0 of node k at index k and out1 at index k + 2^j. If the query encrypts
m(X) = sum_i m_i X^i, output r after J stages encrypts
2^J sum_i m_{2^J i + r} X^(2^J i): a constant 2^J m_r when m has no
coefficient at or above 2^J.

Readings where the paper is silent: the substitution exponents k_j = N/2^j + 1
and the X^(-2^j) factor (one Subs per node: since tau_{k_j}(X^(-2^j)) =
-X^(-2^j), the two substitutions of the two-Subs formulation collapse into one);
the output order above; the key-switching convention (a', b') as written, which
decrypts as b - a s when evk[i] = (u_i, u_i s - tau_k(s) 2^(22 i)); z = 2^22 and
ell = ceil(log2 Q / 22) as in ColTor; evk rows [ell][2][L][N].

Layouts (canonical residues, uint32, NTT form, natural slot order):
    query [2][L][N]                one client's query ciphertext
    evk   [J][ell][2][L][N]        one key per stage
    out   [n_out][2][L][N]         the first n_out of the 2^J outputs
"""

import numpy as np

from .coltor import decompose, gadget_digits
from .ring import intt_negacyclic, ntt_negacyclic, psi_2n


def automorphism_coeffs(a, k: int, q: int) -> np.ndarray:
    """tau_k(a)(X) = a(X^k) mod (X^N + 1, q) on coefficients (k odd)."""
    a = [int(x) for x in a]
    N = len(a)
    out = [0] * N
    for i, ai in enumerate(a):
        e = (i * k) % (2 * N)
        if e < N:
            out[e] = (out[e] + ai) % q
        else:
            out[e - N] = (out[e - N] - ai) % q
    return np.array(out, dtype=np.uint64)


def automorphism_ntt(A, k: int, q: int) -> np.ndarray:
    """tau_k on an NTT-domain polynomial: inverse NTT, substitute, forward NTT."""
    N = len(A)
    psi = psi_2n(q, N)
    return ntt_negacyclic(automorphism_coeffs(intt_negacyclic(A, q, psi), k, q), q, psi)


def monomial_ntt(e: int, q: int, N: int) -> np.ndarray:
    """NTT of X^e for any integer e (X^N = -1, so X^-e = -X^(N-e))."""
    e %= 2 * N
    c = [0] * N
    if e < N:
        c[e] = 1
    else:
        c[e - N] = q - 1
    return ntt_negacyclic(c, q, psi_2n(q, N))


def subs(ct, k: int, evk, primes) -> np.ndarray:
    """Subs(ct, k) with key switching by evk [ell][2][L][N]: ct [2][L][N] -> [2][L][N]."""
    primes = [int(q) for q in primes]
    L = len(primes)
    ct = np.asarray(ct)
    N = ct.shape[-1]
    ell = gadget_digits(primes)
    ta = np.stack([automorphism_ntt(ct[0][l], k, q) for l, q in enumerate(primes)])
    tb = np.stack([automorphism_ntt(ct[1][l], k, q) for l, q in enumerate(primes)])
    digits = decompose(ta, primes, ell)
    out = np.zeros((2, L, N), dtype=np.uint64)
    out[1] = tb
    for i in range(ell):
        for l, q in enumerate(primes):
            d_ntt = ntt_negacyclic([di % q for di in digits[i]], q, psi_2n(q, N))
            for r in range(2):
                row = np.asarray(evk[i][r][l], dtype=np.uint64)
                out[r, l] = (out[r, l] + (d_ntt * row) % np.uint64(q)) % np.uint64(q)
    return out.astype(np.uint32)


def expand_node(ct, j: int, evk_j, primes):
    """One tree node at stage j: (c + t, X^(-2^j) (c - t)) with t = Subs(c, N/2^j + 1)."""
    primes = [int(q) for q in primes]
    ct = np.asarray(ct)
    N = ct.shape[-1]
    t = subs(ct, N // (1 << j) + 1, evk_j, primes).astype(np.int64)
    c = ct.astype(np.int64)
    qv = np.array(primes, dtype=np.int64).reshape(1, -1, 1)
    out0 = ((c + t) % qv).astype(np.uint64)
    diff = ((c - t) % qv).astype(np.uint64)
    out1 = np.empty_like(diff)
    for l, q in enumerate(primes):
        x = monomial_ntt(-(1 << j), q, N)
        for r in range(2):
            out1[r, l] = (diff[r, l] * x) % np.uint64(q)
    return out0.astype(np.uint32), out1.astype(np.uint32)


def expand_query(query, evk, primes, n_out: int) -> np.ndarray:
    """The expansion tree for one client: query [2][L][N], evk [J][ell][2][L][N]
    -> the first n_out (1 <= n_out <= 2^J) outputs [n_out][2][L][N]."""
    J = len(evk)
    if not 1 <= n_out <= (1 << J):
        raise ValueError("n_out must lie in [1, 2^J]")
    level = [np.asarray(query)]
    for j in range(J):
        nxt = [None] * (2 * len(level))
        for k, c in enumerate(level):
            nxt[k], nxt[k + len(level)] = expand_node(c, j, evk[j], primes)
        level = nxt
    return np.stack(level[:n_out])
