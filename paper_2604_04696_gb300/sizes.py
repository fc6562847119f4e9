"""Byte and operation counts of RowSel (host-side arithmetic on shapes only).

Units: one residue is a 32-bit word (Sec. 2.4.1); a polynomial is L limbs of N
residues ("4N points" for the paper's four limbs); a ciphertext is two
polynomials (Sec. 2.2).
"""

WORD = 4


def poly_bytes(N, L):
    return L * N * WORD


def ct_bytes(N, L):
    return 2 * poly_bytes(N, L)


def db_bytes(D0, D1, N, L):
    return D0 * D1 * poly_bytes(N, L)


def query_ct_bytes(B, D0, N, L):
    """Selection ciphertexts of a batch: B clients x D0 ciphertexts."""
    return B * D0 * ct_bytes(N, L)


def out_bytes(B, D1, N, L):
    return B * D1 * ct_bytes(N, L)


def rowsel_algorithmic_bytes(B, D0, D1, N, L):
    """DB read once, selection ciphertexts read once, outputs written once."""
    return db_bytes(D0, D1, N, L) + query_ct_bytes(B, D0, N, L) + out_bytes(B, D1, N, L)


def rowsel_modmacs(B, D0, D1, N, L):
    """Modular multiply-accumulates: (L*N points) x (2B x D0) x (D0 x D1)."""
    return L * N * 2 * B * D0 * D1


def raw_record_bytes(N, log_p):
    """Information content of one plaintext record: N log P bits (Sec. 6)."""
    return N * log_p // 8


def naive_transpose_bytes(B, D0, D1, N, L):
    """Traffic of separate input and output transposes (read + write each)."""
    return 2 * (query_ct_bytes(B, D0, N, L) + out_bytes(B, D1, N, L))
