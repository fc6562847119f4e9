"""A Python model of the GPU NTT schedule of the ciphertext-tree kernels (the
radix-8 rounds, thread-to-set maps, padded shared-memory layout, per-thread
twiddle copies of the bit-reversed rounds, Harvey lazy butterflies with Shoup
products in exact 32-bit arithmetic, and the offset form of the gadget digits),
checked on the CPU against the oracle's transforms and digit routine.

It restates the device code's index and arithmetic rules independently (no code
is shared with the CUDA sources), so that a mistake in the schedule's index
arithmetic, in a lazy-reduction bound or in the bank-conflict claim shows up
here without a GPU.
"""

import numpy as np
import pytest

import oracle
import synth

M32 = (1 << 32) - 1
HALF = 512


def brev(x, bits):
    r = 0
    for i in range(bits):
        r |= ((x >> i) & 1) << (bits - 1 - i)
    return r


def pad(x):
    return x + (x >> 7)


def tables(q, N):
    """fw[k] = (psi^brv(k), Shoup quotient), iv likewise with psi^-1; per-thread
    copies of the twiddles of the bit-reversed rounds."""
    logn = N.bit_length() - 1
    psi = oracle.psi_2n(q, N)
    pinv = pow(psi, q - 2, q)
    sh = lambda w: (w << 32) // q
    fw = [(pow(psi, brev(k, logn), q), 0) for k in range(N)]
    fw = [(w, sh(w)) for w, _ in fw]
    iv = [(pow(pinv, brev(k, logn), q), 0) for k in range(N)]
    iv = [(w, sh(w)) for w, _ in iv]
    S = N // 8
    fwl, ivf = [], []
    for b in range(S):
        i = brev(b, logn - 3)
        fwl.append([fw[S + i], fw[2 * S + 2 * i], fw[2 * S + 2 * i + 1], (0, 0)] + [fw[4 * S + 4 * i + k] for k in range(4)])
        ivf.append([iv[4 * S + 4 * i + k] for k in range(4)] + [iv[2 * S + 2 * i], iv[2 * S + 2 * i + 1], iv[S + i], (0, 0)])
    return fw, iv, fwl, ivf


def shoup_lazy(a, w, ws, q):
    assert 0 <= a <= M32
    r = (a * w - ((a * ws) >> 32) * q) & M32
    assert r < 2 * q                      # the lazy bound the kernels rely on
    return r


def csub(x, c):
    return min(x, (x - c) & M32)


def ct(x, y, w, q):
    """No reduction of its own; the round entry keeps x + 2q and y below 2^32."""
    assert x < 12 * q and y < 12 * q        # at most two levels after the entry
    t = shoup_lazy(y, w[0], w[1], q)
    return (x + t) & M32, (x - t + 2 * q) & M32


def fwd_entry(v, q):
    """Start of a forward round: values below 16q are brought below 8q."""
    for k in range(len(v)):
        assert v[k] < 16 * q
        v[k] = csub(v[k], 8 * q)
        assert v[k] < 8 * q


def gs(x, y, w, q):
    assert x < 2 * q and y < 2 * q
    u = csub((x + y) & M32, 2 * q)
    t = (x - y + 2 * q) & M32
    return u, shoup_lazy(t, w[0], w[1], q)


def fwd_round(v, tw, R, q):
    """tw(r, k) -> twiddle of level r for the pair starting at k."""
    fwd_entry(v, q)
    for r in range(R):
        span = 1 << (R - 1 - r)
        for k in range(1 << R):
            if not k & span:
                v[k], v[k + span] = ct(v[k], v[k + span], tw(r, k), q)


def inv_round(v, tw, R, q):
    for r in range(R):
        span = 1 << r
        for k in range(1 << R):
            if not k & span:
                v[k], v[k + span] = gs(v[k], v[k + span], tw(r, k), q)


def middle_levels(left):
    return 2 if left == 4 else (left if left < 3 else 3)


def set_of(sb, inner, R, N):
    if R == 3 and inner == 8 and N >= 256:
        return (sb >> 5) + (N >> 8) * ((sb >> 3) & 3), sb & 7
    return sb // inner, sb % inner


class Smem:
    """A padded buffer that records, per round, every thread's word addresses."""

    def __init__(self, N):
        self.w = [None] * (N + (N >> 7))
        self.log = []

    def access(self, per_thread):
        self.log.append(per_thread)


def forward(coef, q, N, T, sm):
    fw, _, fwl, _ = T
    logn, S = N.bit_length() - 1, N // 8
    out = [None] * N
    acc = []
    for b in range(S):
        v = [coef[b + k * S] for k in range(8)]
        fwd_round(v, lambda r, k: fw[(1 << r) + (k >> (3 - r))], 3, q)
        addr = [pad(b) + k * S + ((k * S) >> 7) for k in range(8)]
        assert addr == [pad(b + k * S) for k in range(8)]
        for a, x in zip(addr, v):
            sm.w[a] = x
        acc.append(addr)
    sm.access(acc)
    end = logn - 3 if logn >= 6 else logn
    lvl = 3
    while lvl < end:
        R = middle_levels(end - lvl)
        m0, U = 1 << lvl, N >> (lvl + R)
        acc, seen = [], set()
        for b in range(S):
            addrs = []
            for sb in range(b, N >> R, S):
                i, o = set_of(sb, U, R, N)
                base = (i << R) * U + o
                pos = [base + k * U for k in range(1 << R)]
                addr = [pad(base) + k * U + ((k * U) >> 7) for k in range(1 << R)]
                assert addr == [pad(x) for x in pos]
                seen.update(pos)
                v = [sm.w[a] for a in addr]
                fwd_round(v, lambda r, k: fw[(m0 << r) + (i << r) + (k >> (R - r))], R, q)
                for a, x in zip(addr, v):
                    sm.w[a] = x
                addrs += addr
            acc.append(addrs)
        assert len(seen) == N
        sm.access(acc)
        lvl += R
    acc = []
    for b in range(S):
        if logn >= 6:
            i = brev(b, logn - 3)
            addr = [pad(8 * i) + k for k in range(8)]
            w = [sm.w[a] for a in addr]
            t = fwl[b]
            tw = {(0, 0): t[0], (1, 0): t[1], (1, 4): t[2], (2, 0): t[4], (2, 2): t[5], (2, 4): t[6], (2, 6): t[7]}
            fwd_round(w, lambda r, k: tw[(r, k & ~((1 << (3 - r)) - 1))], 3, q)
            for e, k in enumerate([0, 4, 2, 6, 1, 5, 3, 7]):
                out[b + e * S] = w[k]
            acc.append(addr)
        else:
            for e in range(8):
                out[b + e * S] = sm.w[pad(brev(b + e * S, logn))]
    if acc:
        sm.access(acc)
    return out


def inverse(slots, q, N, T, sm):
    _, iv, _, ivf = T
    logn, S = N.bit_length() - 1, N // 8
    ninv = pow(N, q - 2, q)
    ninv_s = (ninv << 32) // q
    acc = []
    for b in range(S):
        i = brev(b, logn - 3)
        v = [slots[b + e * S] for e in (0, 4, 2, 6, 1, 5, 3, 7)]
        if logn >= 6:
            t = ivf[b]
            tw = {(0, 0): t[0], (0, 2): t[1], (0, 4): t[2], (0, 6): t[3], (1, 0): t[4], (1, 4): t[5], (2, 0): t[6]}
            inv_round(v, lambda r, k: tw[(r, k & ~((2 << r) - 1))], 3, q)
        else:
            h0 = N // 2
            inv_round(v, lambda r, k: iv[(h0 >> r) + (i << (2 - r)) + (k >> (r + 1))], 3, q)
        addr = [pad(8 * i) + k for k in range(8)]
        for a, x in zip(addr, v):
            sm.w[a] = x
        acc.append(addr)
    sm.access(acc)
    end = logn - 3 if logn >= 6 else logn
    g = 3
    while g < end:
        R = middle_levels(end - g)
        t0 = 1 << g
        acc = []
        for b in range(S):
            addrs = []
            for sb in range(b, N >> R, S):
                i, o = set_of(sb, t0, R, N)
                base = (i << R) * t0 + o
                addr = [pad(base) + k * t0 + ((k * t0) >> 7) for k in range(1 << R)]
                v = [sm.w[a] for a in addr]
                h0 = N // (2 * t0)
                inv_round(v, lambda r, k: iv[(h0 >> r) + (i << (R - 1 - r)) + (k >> (r + 1))], R, q)
                for a, x in zip(addr, v):
                    sm.w[a] = x
                addrs += addr
            acc.append(addrs)
        sm.access(acc)
        g += R
    out = [None] * N
    acc = []
    for b in range(S):
        addr = [pad(b) + k * S + ((k * S) >> 7) for k in range(8)]
        w = [sm.w[a] for a in addr]
        if logn >= 6:
            inv_round(w, lambda r, k: iv[(4 >> r) + (k >> (r + 1))], 3, q)
        for k in range(8):
            out[b + k * S] = csub(shoup_lazy(w[k], ninv, ninv_s, q), q)
        acc.append(addr)
    sm.access(acc)
    return out


def worst_ways(log):
    """Largest number of distinct words one bank serves in one warp-wide access."""
    worst = 1
    for per_thread in log:
        for w0 in range(0, len(per_thread), 32):
            for a in range(len(per_thread[w0])):
                banks = {}
                for t in per_thread[w0:w0 + 32]:
                    banks.setdefault(t[a] % 32, set()).add(t[a])
                worst = max(worst, max(len(s) for s in banks.values()))
    return worst


@pytest.mark.parametrize("logn", list(range(4, 13)))
def test_schedule_matches_the_oracle_transforms(logn):
    N = 1 << logn
    rng = np.random.default_rng(logn)
    for q in synth.PRIMES_28:
        T = tables(q, N)
        a = [int(x) for x in rng.integers(0, q, N)]
        want = [int(x) for x in oracle.ntt_negacyclic(a, q, oracle.psi_2n(q, N))]
        got = forward(a, q, N, T, Smem(N))
        assert all(x < 14 * q for x in got)   # lazy output range (< 2^32 for q < 2^28)
        assert [x % q for x in got] == want
        # inverse from lazily reduced slot values (< 2q), as the kernels feed it
        lazy = [x + (q if (i % 3 == 0 and x < q) else 0) for i, x in enumerate(want)]
        assert inverse(lazy, q, N, T, Smem(N)) == a


def test_no_bank_conflicts_at_n4096():
    N, q = 4096, synth.PRIMES_28[0]
    T = tables(q, N)
    a = [int(x) for x in np.random.default_rng(0).integers(0, q, N)]
    sm = Smem(N)
    A = forward(a, q, N, T, sm)
    assert worst_ways(sm.log) == 1
    sm = Smem(N)
    inverse([x % q for x in A], q, N, T, sm)
    assert worst_ways(sm.log) == 1


def test_offset_digits_match_the_oracle():
    """y = x + sum_{k < ell-1} (z/2) z^k turns the balanced digits into bit fields."""
    z = 1 << 22
    for primes in (synth.PRIMES_28[:1], synth.PRIMES_28):
        Q = int(np.prod([int(q) for q in primes], dtype=object))
        ell = oracle.gadget_digits(primes)
        O = sum((z // 2) * z ** k for k in range(ell - 1))
        xs = [int(v) for v in np.random.default_rng(1).integers(-(Q // 2) + 1, Q // 2 + 1, 5000)]
        xs += [Q // 2, -(Q // 2) + 1, 0, -1, 1, z // 2, -(z // 2), z // 2 - 1, -(z // 2) - 1]
        for x in xs:
            y = x + O
            d = [((((y % (1 << 64)) >> (22 * i)) & (z - 1)) - z // 2) if i + 1 < ell else (y >> (22 * i))
                 for i in range(ell)]
            assert d == oracle.balanced_digits(x, z, ell)
            assert all(abs(di) < min(primes) for di in d)


def reduce64(x, q):
    """The kernels' Barrett reduction: mu = floor(2^64 / q), qhat = high 64 bits
    of x * mu, r = x - qhat q, one conditional subtraction."""
    mu = ((1 << 64) - 1) // q
    qhat = (x * mu) >> 64
    r = x - qhat * q
    assert 0 <= r < 2 * q            # the bound the single subtraction relies on
    return r - q if r >= q else r


def test_barrett_reduce64_any_64_bit_input():
    rng = np.random.default_rng(5)
    for q in list(synth.PRIMES_28) + [97, 193, (1 << 28) - 57]:
        xs = [0, 1, q - 1, q, 2 * q - 1, (1 << 64) - 1, (1 << 64) - q, ((1 << 64) // q) * q,
              ((1 << 64) // q) * q - 1] + [int(v) for v in rng.integers(0, 1 << 63, 2000, dtype=np.uint64)] + \
             [int(v) << 1 | 1 for v in rng.integers(0, 1 << 63, 2000, dtype=np.uint64)]
        for x in xs:
            assert reduce64(x, q) == x % q


def test_tree_accumulator_bounds():
    """The trees' 64-bit multiply-accumulate: at most 2 ell <= 6 terms, each a lazy
    forward-transform output (< 14q) times a key residue (< q); 14q < 2^32."""
    for q in list(synth.PRIMES_28) + [(1 << 28) - 57]:
        assert 14 * q < 1 << 32
        assert 6 * (14 * q - 1) * (q - 1) < 1 << 63
