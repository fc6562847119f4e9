"""Ring helpers for the RowSel oracle: primes, roots of unity, negacyclic NTT.

Test infrastructure (see the package docstring). These routines exist only so
that the oracle's self-checks can tie the slot-wise product RowSel performs to
the polynomial product it stands for: Sec. 2.4.1 of the GPIR paper states
NTT(a * b) = NTT(a) (.) NTT(b) for the negacyclic ring Z_q[X]/(X^N + 1), which
is what makes RowSel point-wise.

Everything is O(N^2) by definition, with no butterflies: slow and easy to read.
"""

import functools

import numpy as np


def is_prime(n: int) -> bool:
    """Trial division; enough for the <= 32-bit moduli used here."""
    if n < 2:
        return False
    if n % 2 == 0:
        return n == 2
    d = 3
    while d * d <= n:
        if n % d == 0:
            return False
        d += 2
    return True


def ntt_friendly_primes(n: int, bits: int, count: int):
    """The `count` largest primes q < 2**bits with q = 1 (mod 2n), descending.

    q = 1 mod 2n is what a length-n negacyclic NTT needs (a primitive 2n-th
    root of unity exists mod q), Sec. 2.4.1.
    """
    out = []
    q = ((2 ** bits - 1) // (2 * n)) * (2 * n) + 1
    while q >= 2 ** bits:
        q -= 2 * n
    while len(out) < count and q > 2 * n:
        if is_prime(q):
            out.append(q)
        q -= 2 * n
    return out


def _factor(n: int):
    fs, d = [], 2
    while d * d <= n:
        if n % d == 0:
            fs.append(d)
            while n % d == 0:
                n //= d
        d += 1
    if n > 1:
        fs.append(n)
    return fs


def primitive_root(q: int) -> int:
    """Smallest generator of the multiplicative group Z_q^*, q prime."""
    fs = _factor(q - 1)
    g = 2
    while True:
        if all(pow(g, (q - 1) // f, q) != 1 for f in fs):
            return g
        g += 1


def psi_2n(q: int, n: int) -> int:
    """psi = g^((q-1)/2n): a primitive 2n-th root of unity mod q (psi^n = -1)."""
    if (q - 1) % (2 * n) != 0:
        raise ValueError("q must be 1 mod 2n")
    return pow(primitive_root(q), (q - 1) // (2 * n), q)


def _power_table(base: int, count: int, q: int) -> np.ndarray:
    t = np.empty(count, dtype=np.uint64)
    v = 1
    for e in range(count):
        t[e] = v
        v = v * base % q
    return t


def _modmatvec(w: np.ndarray, a: np.ndarray, q: int) -> np.ndarray:
    """(w @ a) mod q with every product reduced before it is summed (no overflow)."""
    q64 = np.uint64(q)
    out = np.zeros(w.shape[0], dtype=np.uint64)
    for j in range(w.shape[1]):
        out = (out + (w[:, j] * np.uint64(a[j])) % q64) % q64
    return out


@functools.lru_cache(maxsize=8)
def _ntt_matrix(q: int, psi: int, n: int, inverse: bool) -> np.ndarray:
    """W[s][j] = psi^((2s+1) j) (forward) or W[j][s] = psi^-((2s+1) j) (inverse), mod q.
    Memoised: the definition's matrix does not depend on the data."""
    base = pow(psi, q - 2, q) if inverse else psi
    pw = _power_table(base, 2 * n, q)
    r = np.arange(n, dtype=np.int64)[:, None]
    c = np.arange(n, dtype=np.int64)[None, :]
    return pw[((2 * c + 1) * r) % (2 * n)] if inverse else pw[((2 * r + 1) * c) % (2 * n)]


def ntt_negacyclic(a, q: int, psi: int) -> np.ndarray:
    """Natural-order negacyclic NTT by definition: A_s = sum_j a_j psi^((2s+1) j) mod q."""
    a = np.asarray(a, dtype=np.uint64)
    return _modmatvec(_ntt_matrix(q, psi, a.shape[0], False), a, q)


def intt_negacyclic(A, q: int, psi: int) -> np.ndarray:
    """Inverse of ntt_negacyclic: a_j = n^-1 sum_s A_s psi^-((2s+1) j) mod q."""
    A = np.asarray(A, dtype=np.uint64)
    n = A.shape[0]
    a = _modmatvec(_ntt_matrix(q, psi, n, True), A, q)
    n_inv = pow(n, q - 2, q)
    return (a * np.uint64(n_inv)) % np.uint64(q)


def schoolbook_negacyclic(a, b, q: int) -> np.ndarray:
    """c = a * b in Z_q[X]/(X^n + 1) by the schoolbook rule X^n = -1 (Python ints)."""
    a = [int(x) for x in a]
    b = [int(x) for x in b]
    n = len(a)
    c = [0] * n
    for i in range(n):
        ai = a[i]
        if ai == 0:
            continue
        for j in range(n):
            k = i + j
            if k < n:
                c[k] += ai * b[j]
            else:
                c[k - n] -= ai * b[j]
    return np.array([x % q for x in c], dtype=np.uint64)
