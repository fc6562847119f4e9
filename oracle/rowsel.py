"""RowSel by its plain definition (test infrastructure; see the package docstring).

GPIR paper, Sec. 2.2 (RowSel) and the GEMM form in Sec. 2.3:
    M_out[p, m, n] = sum_k M_in0[p, m, k] * M_in1[p, k, n],
with p the 4N NTT points (here L limbs x N slots), m the 2 polynomials of a
ciphertext (2 * batch with batching, Sec. 5.1.1), k the D0 database rows and
n the D1 database columns. Each selection ciphertext i is multiplied point-wise
with database row i and the products are summed over the rows, mod the limb's
prime.

Array layouts (canonical residues, uint32):
    ct  [B][D0][2][L][T]   ciphertext i of client c, polynomial r, limb l, slot t
    db  [D0][D1][L][T]     NTT-form plaintext DB[i][j]
    out [B][D1][2][L][T]   output ciphertext j of client c
T may be any subset of the N slots (slot-wise independence), so callers can
evaluate a sample of slots.
"""

import numpy as np


def rowsel(ct, db, primes) -> np.ndarray:
    """out[c][j][r][l][t] = ( sum_i (ct[c][i][r][l][t] * db[i][j][l][t] mod q_l) ) mod q_l."""
    ct = np.asarray(ct)
    db = np.asarray(db)
    B, D0, two, L, T = ct.shape
    if two != 2:
        raise ValueError("a ciphertext has exactly two polynomials")
    if db.shape[0] != D0 or db.shape[2] != L or db.shape[3] != T:
        raise ValueError("ct / db shapes disagree")
    if len(primes) != L:
        raise ValueError("one prime per limb")
    D1 = db.shape[1]
    out = np.empty((B, D1, 2, L, T), dtype=np.uint32)
    for l in range(L):
        q = np.uint64(primes[l])
        acc = np.zeros((B, D1, 2, T), dtype=np.uint64)   # < D0 * q, far below 2^64
        for i in range(D0):
            sel = ct[:, i, :, l, :].astype(np.uint64)     # [B][2][T]: selection ct i
            row = db[i, :, l, :].astype(np.uint64)         # [D1][T]:   DB row i
            acc += (sel[:, None, :, :] * row[None, :, None, :]) % q
        out[:, :, :, l, :] = (acc % q).astype(np.uint32)
    return out


def rowsel_output(ct, db, primes, c: int, j: int, r: int, l: int, t: int) -> int:
    """One output residue out[c][j][r][l][t], summed with Python integers."""
    q = int(primes[l])
    d0 = ct.shape[1]
    s = 0
    for i in range(d0):
        s += int(ct[c, i, r, l, t]) * int(db[i, j, l, t])
    return s % q


def rlwe_decrypt_ntt(out_a, out_b, s, q: int) -> np.ndarray:
    """Noiseless RLWE phase in the NTT domain: b - a (.) s mod q (slot-wise)."""
    q64 = np.uint64(q)
    a = np.asarray(out_a, dtype=np.uint64)
    b = np.asarray(out_b, dtype=np.uint64)
    s = np.asarray(s, dtype=np.uint64)
    return ((b + q64 - (a * s) % q64) % q64).astype(np.uint32)
