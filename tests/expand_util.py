"""Toy ExpandQuery inputs with a known answer (client-side key material, not
part of ExpandQuery), shared by the oracle pins and the GPU parity tests.

The automorphism here is the NTT-domain slot permutation: slot s of a
polynomial holds its value at psi^(2s+1), so tau_k moves the value at slot s'
to slot s where 2s'+1 = (2s+1) k (mod 2N). The oracle computes tau_k through
the coefficients instead, so the two are independent formulations.
"""

import numpy as np

import oracle
import synth

TAG_EVK = synth.TAG_EVK
TAG_QUERY = synth.TAG_QUERY
TAG_MESSAGE = synth.TAG_MESSAGE


def slot_perm(N: int, k: int) -> np.ndarray:
    """src[s] = s' with 2s'+1 = (2s+1) k mod 2N: tau_k(A)[s] = A[src[s]]."""
    s = np.arange(N, dtype=np.int64)
    return (((2 * s + 1) * k) % (2 * N) - 1) // 2


def toy_evk(seed: int, stage: int, k: int, s, L: int, N: int, primes, ell: int, log_base: int = 22):
    """Noiseless toy key-switching key from tau_k(s) to s, NTT domain:
    evk[i] = (u_i, u_i (.) s - tau_k(s) g_i), g_i = 2^(log_base i) mod q.
    Returns [ell][2][L][N] uint32."""
    u = synth.uniform_residues(seed, TAG_EVK, (stage + 1, ell, L, N), primes, limb_axis=2)[stage].astype(np.uint64)
    s = np.asarray(s, dtype=np.uint64)
    perm = slot_perm(N, k)
    out = np.empty((ell, 2, L, N), dtype=np.uint32)
    for l in range(L):
        q = int(primes[l])
        ts = s[l][perm]
        for i in range(ell):
            g = np.uint64(pow(2, log_base * i, q))
            out[i, 0, l] = u[i, l].astype(np.uint32)
            out[i, 1, l] = ((u[i, l] * s[l] + np.uint64(q) - (ts * g) % np.uint64(q)) % np.uint64(q)).astype(np.uint32)
    return out


def toy_expand_inputs(seed: int, J: int, L: int, N: int, primes, ell: int, msg_bound: int = 1 << 20):
    """A toy query encrypting a random message polynomial m (coefficients in
    [0, msg_bound)) and the J stage keys. Returns (query [2][L][N],
    evk [J][ell][2][L][N], s [L][N], m [N] as Python ints)."""
    s = synth.uniform_residues(seed, synth.TAG_SECRET, (L, N), primes, limb_axis=0)
    a = synth.uniform_residues(seed, TAG_QUERY, (L, N), primes, limb_axis=0).astype(np.uint64)
    m = [int(x) % msg_bound for x in synth.uniform_u64(seed, TAG_MESSAGE, 0, N)]
    query = np.empty((2, L, N), dtype=np.uint32)
    for l in range(L):
        q = int(primes[l])
        M = oracle.ntt_negacyclic([x % q for x in m], q, oracle.psi_2n(q, N))
        query[0, l] = a[l].astype(np.uint32)
        query[1, l] = ((a[l] * s[l].astype(np.uint64) + M) % np.uint64(q)).astype(np.uint32)
    evk = np.stack([toy_evk(seed, j, N // (1 << j) + 1, s, L, N, primes, ell) for j in range(J)]) if J else \
        np.zeros((0, ell, 2, L, N), dtype=np.uint32)
    return query, evk, s, m


def phase_coeffs(ct, s, primes):
    """Coefficients of b - a (.) s (noiseless toy decryption), per limb, as lists."""
    out = []
    for l, q in enumerate(primes):
        q = int(q)
        a = np.asarray(ct[0][l], dtype=np.uint64)
        b = np.asarray(ct[1][l], dtype=np.uint64)
        ph = (b + np.uint64(q) - (a * np.asarray(s[l], dtype=np.uint64)) % np.uint64(q)) % np.uint64(q)
        out.append([int(x) for x in oracle.intt_negacyclic(ph, q, oracle.psi_2n(q, len(ph)))])
    return out


def expected_output_coeffs(m, J: int, r: int, N: int, primes):
    """Coefficients of 2^J sum_i m_{2^J i + r} X^(2^J i), per limb."""
    out = []
    for q in primes:
        c = [0] * N
        for i in range(0, N, 1 << J):
            if i + r < N:
                c[i] = ((1 << J) * m[i + r]) % int(q)
        out.append(c)
    return out
