"""Counter-based SplitMix64 residues and the workload shapes (no RowSel arithmetic)."""

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
TAGMUL = 0xD1B54A32D192ED03
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

TAG_DB = 1        # database residues
TAG_CT = 2        # selection-ciphertext residues
TAG_SECRET = 3    # toy RLWE secret
TAG_MASK = 4      # toy RLWE uniform "a" polynomials
TAG_RGSW = 5      # toy RGSW uniform "a" polynomials (ColTor inputs)
TAG_COLTOR = 6    # toy RLWE uniform "a" polynomials of ColTor's input ciphertexts
TAG_RECORD = 7    # records (plaintext polynomials) those ciphertexts encrypt
TAG_EVK = 8       # toy evaluation-key uniform polynomials (ExpandQuery inputs)
TAG_QUERY = 9     # query ciphertexts (ExpandQuery inputs)
TAG_MESSAGE = 10  # toy query message coefficients

# The two largest primes below 2^28 that are 1 mod 8192 (so NTT-friendly for
# every N <= 4096): 0xFFF0001 and 0xFFEE001.
PRIMES_28 = (268369921, 268361729)


def mix64(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * M1) & MASK64
    z = ((z ^ (z >> 27)) * M2) & MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, tag: int) -> int:
    return mix64(((seed * GAMMA) ^ ((tag + 1) * TAGMUL)) & MASK64)


def _mix64_np(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(M1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(M2)
    return z ^ (z >> np.uint64(31))


def uniform_u64(seed: int, tag: int, start: int, count: int) -> np.ndarray:
    """value(i) for i in [start, start + count), as uint64."""
    key = np.uint64(stream_key(seed, tag))
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64_np(key + idx * np.uint64(GAMMA))


def uniform_residues(seed: int, tag: int, shape, primes, limb_axis: int,
                     chunk: int = 1 << 24) -> np.ndarray:
    """uint32 array of `shape`; element at flat index f is value(f) mod q_l,
    l the element's index along `limb_axis`."""
    shape = tuple(int(s) for s in shape)
    total = int(np.prod(shape)) if shape else 1
    out = np.empty(total, dtype=np.uint32)
    # limb of each flat index: (f // inner) % L
    L = shape[limb_axis]
    inner = int(np.prod(shape[limb_axis + 1:])) if limb_axis + 1 < len(shape) else 1
    qs = np.asarray(primes, dtype=np.uint64)
    if len(qs) != L:
        raise ValueError("one prime per limb")
    for s in range(0, total, chunk):
        n = min(chunk, total - s)
        v = uniform_u64(seed, tag, s, n)
        limb = (np.arange(s, s + n, dtype=np.int64) // inner) % L
        out[s:s + n] = (v % qs[limb]).astype(np.uint32)
    return out.reshape(shape)


def ct_tensor(seed: int, B: int, D0: int, L: int, N: int, primes) -> np.ndarray:
    """Selection ciphertexts [B][D0][2][L][N], uniform residues."""
    return uniform_residues(seed, TAG_CT, (B, D0, 2, L, N), primes, limb_axis=3)


def db_tensor(seed: int, D0: int, D1: int, L: int, N: int, primes) -> np.ndarray:
    """NTT-form database [D0][D1][L][N], uniform residues."""
    return uniform_residues(seed, TAG_DB, (D0, D1, L, N), primes, limb_axis=2)


def toy_rlwe_selection(seed: int, D0: int, L: int, N: int, primes, istar: int):
    """Noiseless toy RLWE one-hot query in the NTT domain, for serving checks.

    ct_i = (a_i, a_i (.) s + [i == istar] * 1) mod q, with a_i and s uniform.
    (The NTT of the constant polynomial 1 is the all-ones vector.)
    Returns (ct [D0][2][L][N] uint32, s [L][N] uint32).
    This is query encoding on the client side, not RowSel.
    """
    s = uniform_residues(seed, TAG_SECRET, (L, N), primes, limb_axis=0).astype(np.uint64)
    a = uniform_residues(seed, TAG_MASK, (D0, L, N), primes, limb_axis=1).astype(np.uint64)
    ct = np.empty((D0, 2, L, N), dtype=np.uint32)
    for l in range(L):
        q = np.uint64(primes[l])
        b = (a[:, l, :] * s[l][None, :]) % q
        b[istar] = (b[istar] + np.uint64(1)) % q
        ct[:, 0, l, :] = a[:, l, :].astype(np.uint32)
        ct[:, 1, l, :] = b.astype(np.uint32)
    return ct, s.astype(np.uint32)


def toy_rgsw(seed: int, stage: int, m: int, s, L: int, N: int, primes, ell: int, log_base: int = 22):
    """Noiseless toy RGSW encryption of the bit m under secret s (NTT domain), for
    ColTor inputs: rows i < ell are (a_i + m g_i, a_i (.) s), rows ell + i are
    (a'_i, a'_i (.) s + m g_i), with g_i = 2^(log_base i) mod q_l a constant
    polynomial (its NTT is the constant vector). Returns [2 ell][2][L][N] uint32.
    This is key material the client makes, not part of ColTor.
    """
    a = uniform_residues(seed, TAG_RGSW, (stage + 1, 2 * ell, L, N), primes, limb_axis=2)[stage].astype(np.uint64)
    s = np.asarray(s, dtype=np.uint64)
    out = np.empty((2 * ell, 2, L, N), dtype=np.uint32)
    for l in range(L):
        q = np.uint64(primes[l])
        for row in range(2 * ell):
            i = row % ell
            g = np.uint64(pow(2, log_base * i, int(primes[l])) * int(m) % int(primes[l]))
            ar = a[row, l]
            c0 = (ar + g) % q if row < ell else ar
            c1 = (ar * s[l]) % q if row < ell else ((ar * s[l]) % q + g) % q
            out[row, 0, l] = c0.astype(np.uint32)
            out[row, 1, l] = c1.astype(np.uint32)
    return out


def toy_coltor_inputs(seed: int, D1: int, L: int, N: int, primes, jstar: int, ell: int, log_base: int = 22):
    """ColTor inputs for one client with a known answer: D1 noiseless toy RLWE
    ciphertexts ct_j = (a_j, a_j (.) s + R_j) of random records R_j (NTT domain),
    and one toy RGSW encryption of each bit of jstar (least significant first).
    Returns (ct [D1][2][L][N], rgsw [log2 D1][2 ell][2][L][N], s [L][N], R [D1][L][N])."""
    stages = max(0, int(D1).bit_length() - 1)
    s = uniform_residues(seed, TAG_SECRET, (L, N), primes, limb_axis=0)
    a = uniform_residues(seed, TAG_COLTOR, (D1, L, N), primes, limb_axis=1).astype(np.uint64)
    rec = uniform_residues(seed, TAG_RECORD, (D1, L, N), primes, limb_axis=1)
    ct = np.empty((D1, 2, L, N), dtype=np.uint32)
    for l in range(L):
        q = np.uint64(primes[l])
        ct[:, 0, l] = a[:, l].astype(np.uint32)
        ct[:, 1, l] = ((a[:, l] * s[l].astype(np.uint64)) % q + rec[:, l].astype(np.uint64)) % q
    rgsw = np.stack([toy_rgsw(seed, st, (jstar >> st) & 1, s, L, N, primes, ell, log_base)
                     for st in range(stages)]) if stages else np.zeros((0, 2 * ell, 2, L, N), np.uint32)
    return ct, rgsw, s, rec


# Workloads of the GPIR RowSel study on one GB300 (synthetic, uniform residues).
CONFIGS = {
    "c1_plain": dict(N=2048, L=1, D0=16, D1=16, B=1, seed=0),
    "c2_rowsel": dict(N=4096, L=2, D0=256, D1=64, B=32, seed=1),
    "c3_sweep": dict(N=4096, L=2, D0=256, D1=64, B=(1, 8, 32, 128, 256), seed=2),
    "c4_large": dict(N=4096, L=2, D0=1024, D1=128, B=128, seed=3),
    "c5_serving": dict(N=4096, L=2, dbs=((256, 64), (512, 64), (1024, 128)), seed=4),
}


def config_shapes(name: str):
    c = dict(CONFIGS[name])
    c["primes"] = PRIMES_28[:c["L"]]
    return c


def residues_at(seed: int, tag: int, flat_idx, limb, primes) -> np.ndarray:
    """value(f) mod q_limb for arbitrary flat indices f (random access into a
    tensor generated by uniform_residues with the same seed and tag)."""
    f = np.asarray(flat_idx, dtype=np.uint64)
    v = uniform_u64_at(seed, tag, f)
    qs = np.asarray(primes, dtype=np.uint64)[np.asarray(limb, dtype=np.int64)]
    return (v % qs).astype(np.uint32)


def uniform_u64_at(seed: int, tag: int, flat_idx) -> np.ndarray:
    key = np.uint64(stream_key(seed, tag))
    f = np.asarray(flat_idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64_np(key + (f + np.uint64(1)) * np.uint64(GAMMA))


def ct_slots(seed: int, B: int, D0: int, L: int, N: int, primes, slots) -> np.ndarray:
    """ct_tensor(...)[..., l, t] for the given (l, t) slot pairs: [B][D0][2][S]."""
    c = np.arange(B)[:, None, None, None]
    i = np.arange(D0)[None, :, None, None]
    r = np.arange(2)[None, None, :, None]
    ls = np.array([s[0] for s in slots])[None, None, None, :]
    ts = np.array([s[1] for s in slots])[None, None, None, :]
    f = (((c * D0 + i) * 2 + r) * L + ls) * N + ts
    return residues_at(seed, TAG_CT, f, np.broadcast_to(ls, f.shape), primes)


def db_slots(seed: int, D0: int, D1: int, L: int, N: int, primes, slots) -> np.ndarray:
    """db_tensor(...)[..., l, t] for the given (l, t) slot pairs: [D0][D1][S]."""
    i = np.arange(D0)[:, None, None]
    j = np.arange(D1)[None, :, None]
    ls = np.array([s[0] for s in slots])[None, None, :]
    ts = np.array([s[1] for s in slots])[None, None, :]
    f = ((i * D1 + j) * L + ls) * N + ts
    return residues_at(seed, TAG_DB, f, np.broadcast_to(ls, f.shape), primes)
