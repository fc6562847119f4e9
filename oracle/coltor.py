"""ColTor by its definition (test infrastructure; see the package docstring).

GPIR paper, Sec. 2.2 ("ColTor") and Sec. 2.5.1 (the steps of an external
product). ColTor is a binary tournament over RowSel's D1 output ciphertexts
with log2(D1) stages. Each tree node takes two ciphertexts and returns one,
through an external product with the stage's RGSW ciphertext:

    node(ct_lo, ct_hi, RGSW(b)) = ct_lo + RGSW(b) [x] (ct_hi - ct_lo)

so that the node selects ct_hi when b = 1 and ct_lo when b = 0 (in what the
ciphertexts decrypt to). Stage s pairs the stage's inputs (2k, 2k+1) and uses
the RGSW ciphertext of bit s of the column index, least significant bit first.

External product RGSW [x] ct, ct = (c_0, c_1) in the NTT domain (Sec. 2.5.1):
  1. inverse NTT of c_0 and c_1, limb by limb;
  2. Dcp: each coefficient is rebuilt from its L residues (CRT) as an integer
     x in [0, Q), Q = prod q_l, centred to (-Q/2, Q/2], and split into
     balanced base-z digits x = sum_{i<ell} d_i z^i, d_i in [-z/2, z/2);
  3. forward NTT of the 2 ell digit polynomials (digits reduced mod each q_l);
  4. multiply-accumulate with the RGSW rows:
         out_r = sum_{p in {0,1}} sum_{i < ell} NTT(d_{p,i}) (.) rgsw[p ell + i][r],  r in {0, 1}.

Readings where the paper is silent: z = 2^22 (the paper's base) and
ell = ceil(log2(Q) / 22); the pairing order and bit order above; RGSW rows
ordered (polynomial p, digit i) as [2 ell][2][L][N].

Layouts (canonical residues, uint32, NTT form, natural slot order):
    ct    [D1][2][L][N]                  RowSel's output for one client
    rgsw  [log2 D1][2 ell][2][L][N]      one RGSW ciphertext per stage
    out   [2][L][N]
"""

import numpy as np

from .ring import intt_negacyclic, ntt_negacyclic, psi_2n

GADGET_LOG_BASE = 22


def gadget_digits(primes) -> int:
    """ell = ceil(log2 Q / 22) for Q = prod(primes)."""
    Q = 1
    for q in primes:
        Q *= int(q)
    bits = (Q - 1).bit_length()
    return -(-bits // GADGET_LOG_BASE)


def crt_centered(residues, primes) -> list:
    """Integers x in (-Q/2, Q/2] with x = residues[l] (mod primes[l]), one per
    coefficient (residues: [L][N]). Plain CRT with Python integers."""
    primes = [int(q) for q in primes]
    Q = 1
    for q in primes:
        Q *= q
    L, N = len(primes), len(residues[0])
    out = []
    for j in range(N):
        x = 0
        for l in range(L):
            Ml = Q // primes[l]
            x += int(residues[l][j]) * Ml * pow(Ml, -1, primes[l])
        x %= Q
        if x > Q // 2:
            x -= Q
        out.append(x)
    return out


def balanced_digits(x: int, z: int, ell: int) -> list:
    """d_0..d_{ell-1} with x = sum d_i z^i and d_i in [-z/2, z/2) (the last
    digit takes what is left)."""
    d = []
    for i in range(ell):
        if i == ell - 1:
            d.append(x)
            break
        r = x % z
        if r >= z // 2:
            r -= z
        d.append(r)
        x = (x - r) // z
    return d


def decompose(poly_ntt, primes, ell: int):
    """Dcp of one NTT-domain polynomial [L][N]: inverse NTT, CRT, balanced
    digits. Returns digits[ell][N] as Python integers."""
    primes = [int(q) for q in primes]
    L, N = len(primes), len(poly_ntt[0])
    coef = [intt_negacyclic(poly_ntt[l], primes[l], psi_2n(primes[l], N)) for l in range(L)]
    xs = crt_centered(coef, primes)
    z = 1 << GADGET_LOG_BASE
    digits = [[0] * N for _ in range(ell)]
    for j, x in enumerate(xs):
        for i, di in enumerate(balanced_digits(x, z, ell)):
            digits[i][j] = di
    return digits


def external_product(rgsw, ct, primes) -> np.ndarray:
    """RGSW [x] ct, both NTT domain: rgsw [2 ell][2][L][N], ct [2][L][N] -> [2][L][N]."""
    primes = [int(q) for q in primes]
    L = len(primes)
    ct = np.asarray(ct)
    N = ct.shape[-1]
    ell = gadget_digits(primes)
    out = np.zeros((2, L, N), dtype=np.uint64)
    for p in range(2):
        digits = decompose(ct[p], primes, ell)
        for i in range(ell):
            for l, q in enumerate(primes):
                d_ntt = ntt_negacyclic([di % q for di in digits[i]], q, psi_2n(q, N))
                for r in range(2):
                    row = np.asarray(rgsw[p * ell + i][r][l], dtype=np.uint64)
                    out[r, l] = (out[r, l] + (d_ntt * row) % np.uint64(q)) % np.uint64(q)
    return out.astype(np.uint32)


def cmux(rgsw, ct_lo, ct_hi, primes) -> np.ndarray:
    """ct_lo + RGSW [x] (ct_hi - ct_lo), the tree node of ColTor."""
    primes = [int(q) for q in primes]
    lo = np.asarray(ct_lo, dtype=np.int64)
    hi = np.asarray(ct_hi, dtype=np.int64)
    qv = np.array(primes, dtype=np.int64).reshape(1, -1, 1)
    diff = ((hi - lo) % qv).astype(np.uint32)
    ep = external_product(rgsw, diff, primes).astype(np.int64)
    return ((lo + ep) % qv).astype(np.uint32)


def coltor(ct, rgsw, primes) -> np.ndarray:
    """The tournament over one client's D1 ciphertexts: ct [D1][2][L][N],
    rgsw [log2 D1][2 ell][2][L][N] -> [2][L][N]."""
    level = [np.asarray(c) for c in ct]
    D1 = len(level)
    if D1 & (D1 - 1):
        raise ValueError("D1 must be a power of two")
    s = 0
    while len(level) > 1:
        level = [cmux(rgsw[s], level[2 * k], level[2 * k + 1], primes) for k in range(len(level) // 2)]
        s += 1
    return level[0]
