"""CPU models of the exact arithmetic of the RowSel paths, checked against the
oracle: the tensor-core fused kernel (fp16 digits, 512-row fp32 groups), the
two-pass kernel (256-row groups, magic-number conversion), the INT8 path
(unsigned byte limbs, int32 diagonal sums folded every 8192 rows) and the
CUDA-core path (64-bit sums reduced every 256 rows).

The tensor-core path (tcgen05 .kind::f16) rests on an exactness argument:
  - each residue x < 2^28 splits into balanced base-256 digits, byte u of
    x + 0x808080 minus 128 for u < 3 and byte 3 as is, so that
    x = sum_u d_u 2^(8u) with d_0..d_2 in [-128, 127] and d_3 in [0, 16],
    every digit exactly an fp16;
  - a digit product is at most 2^14 in magnitude, so a sum over a group of
    512 rows is at most 2^23 and every partial sum is an integer an fp32
    accumulator holds exactly, in any order;
  - the group sums D_uv are recombined as sum_uv D_uv (2^(8(u+v)) mod q) in
    64-bit integers (< 2^55 per group), up to 8 groups are added (< 2^58), and
    one Barrett reduction of the sum plus off58 (the smallest multiple of q not
    below 2^58) finishes each flush.
This model restates those steps with numpy (float32 group products, int64
recombination) without any code of the CUDA path, and checks the result
against the oracle; a negative control shows the float32 sums failing once the
group bound is broken.
"""

import numpy as np
import pytest

import oracle
import synth

PRIMES = synth.PRIMES_28
GROUP = 512
FLUSH = 8


def digits(x):
    """[..., 4] balanced base-256 digits of x (uint32 array, x < 2^28)."""
    xp = x.astype(np.int64) + 0x808080
    d = np.stack([(xp >> (8 * u)) & 0xFF for u in range(4)], axis=-1)
    d[..., :3] -= 128
    return d


def tc_model_rowsel(ct, db, primes):
    """ct [B][D0][2][L][T], db [D0][D1][L][T] -> [B][D1][2][L][T] through the digit model."""
    ct = np.asarray(ct)
    db = np.asarray(db)
    B, D0, _, L, T = ct.shape
    D1 = db.shape[1]
    out = np.zeros((B, D1, 2, L, T), dtype=np.uint64)
    for l, q in enumerate(primes):
        q = int(q)
        c = np.array([pow(2, 8 * s, q) for s in range(7)], dtype=np.int64)
        off58 = -(-(1 << 58) // q) * q
        for t in range(T):
            a = digits(ct[:, :, :, l, t].transpose(0, 2, 1).reshape(2 * B, D0))     # [2B][D0][4]
            bd = digits(db[:, :, l, t])                                               # [D0][D1][4]
            res = np.zeros((2 * B, D1), dtype=np.uint64)
            acc = np.zeros((2 * B, D1), dtype=np.int64)
            groups = 0
            for g0 in range(0, D0, GROUP):
                g1 = min(D0, g0 + GROUP)
                for u in range(4):
                    A = a[:, g0:g1, u].astype(np.float32)
                    for v in range(4):
                        Bm = bd[g0:g1, :, v].astype(np.float32)
                        D = (A @ Bm).astype(np.float64)               # fp32 products and sums
                        assert np.all(np.abs(D) <= 2 ** 23)
                        acc += np.rint(D).astype(np.int64) * c[u + v]
                groups += 1
                if groups == FLUSH or g1 == D0:
                    assert np.all(np.abs(acc) < 2 ** 58)
                    r = ((acc + off58).astype(np.uint64) % np.uint64(q))
                    res = (res + r) % np.uint64(q)
                    acc[:] = 0
                    groups = 0
            out[:, :, :, l, t] = res.reshape(B, 2, D1).transpose(0, 2, 1)
    return out.astype(np.uint32)


def test_digit_split_reconstructs_and_fits_fp16():
    rng = np.random.default_rng(1)
    for q in PRIMES:
        xs = np.concatenate([rng.integers(0, q, 20000), [0, 1, 127, 128, 255, 256, 0x7F7F7F, 0x808080, q - 1,
                                                         (1 << 28) - 1]]).astype(np.uint32)
        d = digits(xs)
        assert np.array_equal((d * (256 ** np.arange(4))).sum(axis=-1), xs.astype(np.int64))
        assert d[..., :3].min() >= -128 and d[..., :3].max() <= 127
        assert d[..., 3].min() >= 0 and d[..., 3].max() <= 16
        assert np.array_equal(d.astype(np.float16).astype(np.int64), d)      # exact fp16 values


def test_group_sums_are_exact_in_fp32_at_the_bound():
    """The worst case of a 512-row group (all digit products 2^14) and random
    signed digits: float32 sums equal the integer sums."""
    a = np.full((4, GROUP), -128, dtype=np.int64)
    b = np.full((GROUP, 4), -128, dtype=np.int64)
    assert np.array_equal((a.astype(np.float32) @ b.astype(np.float32)).astype(np.int64), a @ b)
    rng = np.random.default_rng(2)
    a = rng.integers(-128, 128, (64, GROUP))
    b = rng.integers(-128, 128, (GROUP, 64))
    assert np.array_equal((a.astype(np.float32) @ b.astype(np.float32)).astype(np.int64), a @ b)


def test_group_bound_is_needed():
    """Negative control: over 8 x 512 rows of odd products a float32 running sum
    passes 2^24 and drops low bits."""
    a = np.full(8 * GROUP, 127, dtype=np.int64)
    b = np.full(8 * GROUP, 127, dtype=np.int64)
    acc = np.float32(0)
    for x, y in zip(a, b):
        acc = np.float32(acc + np.float32(x * y))
    assert int(acc) != int((a * b).sum())


@pytest.mark.parametrize("shape", [(2, 5000, 7, 2, 3), (1, 513, 4, 1, 2), (3, 64, 5, 2, 4)])
def test_model_equals_oracle(shape):
    """Random residues and the all-(q-1) worst case, D0 across several groups and flushes."""
    B, D0, D1, L, T = shape
    primes = PRIMES[:L]
    ct = synth.uniform_residues(61 + D0, synth.TAG_CT, (B, D0, 2, L, T), primes, limb_axis=3)
    db = synth.uniform_residues(62 + D0, synth.TAG_DB, (D0, D1, L, T), primes, limb_axis=2)
    assert np.array_equal(tc_model_rowsel(ct, db, primes), oracle.rowsel(ct, db, primes))
    qm = np.array(primes, dtype=np.uint32)
    ct_w = np.broadcast_to(qm[None, None, None, :, None] - 1, ct.shape).copy()
    db_w = np.broadcast_to(qm[None, None, :, None] - 1, db.shape).copy()
    assert np.array_equal(tc_model_rowsel(ct_w, db_w, primes), oracle.rowsel(ct_w, db_w, primes))


MAGIC = 0x4B400000          # bit pattern of 1.5 * 2^23 in fp32
GROUP2 = 256                # rows per exact group in the two-pass kernel


def magic_bits(D):
    """Bit pattern of fp32(D) + 1.5 * 2^23, as the two-pass epilogue forms it."""
    return (np.asarray(D, dtype=np.float32) + np.float32(12582912.0)).view(np.int32).astype(np.int64)


def test_magic_conversion_exact_within_2_22():
    """fp32 D + 1.5 * 2^23 has bit pattern MAGIC + D exactly for |D| <= 2^22,
    the bound of a 256-row group of digit products (256 * 2^14)."""
    rng = np.random.default_rng(3)
    D = np.concatenate([rng.integers(-(1 << 22), (1 << 22) + 1, 100000), [0, 1, -1, 1 << 22, -(1 << 22)]])
    assert np.array_equal(magic_bits(D) - MAGIC, D)
    # negative control: one past the bound the spacing is 2 (above) or the scale changes (below)
    assert magic_bits((1 << 22) + 1) - MAGIC != (1 << 22) + 1
    assert magic_bits(-(1 << 22) - 1) - MAGIC != -(1 << 22) - 1


def test_two_pass_sum_bound():
    """sum over the 16 digit pairs of bits * c stays below 2^63 for the real
    primes: bits <= MAGIC + 2^22 and c < q."""
    for q in PRIMES:
        assert 16 * (MAGIC + (1 << 22)) * (int(q) - 1) < 1 << 63


def tc_model_rowsel_two_pass(ct, db, primes):
    """The two-pass epilogue: 256-row groups, magic conversion, kfix removed,
    one Barrett reduction (offset by a multiple of q >= 2^55) per group."""
    ct = np.asarray(ct)
    db = np.asarray(db)
    B, D0, _, L, T = ct.shape
    D1 = db.shape[1]
    out = np.zeros((B, D1, 2, L, T), dtype=np.uint64)
    for l, q in enumerate(primes):
        q = int(q)
        c = [pow(2, 8 * s, q) for s in range(7)]
        kfix = MAGIC * sum(c[u + v] for u in range(4) for v in range(4))
        off = -(-(1 << 55) // q) * q
        for t in range(T):
            a = digits(ct[:, :, :, l, t].transpose(0, 2, 1).reshape(2 * B, D0))
            bd = digits(db[:, :, l, t])
            res = np.zeros((2 * B, D1), dtype=object)
            for g0 in range(0, D0, GROUP2):
                g1 = min(D0, g0 + GROUP2)
                keep = np.zeros((2 * B, D1), dtype=object)
                for u in range(4):
                    for v in range(4):
                        Dm = a[:, g0:g1, u].astype(np.float32) @ bd[g0:g1, :, v].astype(np.float32)
                        assert np.all(np.abs(Dm) <= 1 << 22)
                        keep = keep + magic_bits(Dm).astype(object) * c[u + v]
                x = keep - kfix + off
                assert all(0 <= int(v) < 1 << 64 for v in np.ravel(x))
                res = (res + x % q) % q
            out[:, :, :, l, t] = res.astype(np.uint64).reshape(B, 2, D1).transpose(0, 2, 1)
    return out.astype(np.uint32)


@pytest.mark.parametrize("shape", [(2, 600, 5, 2, 2), (1, 256, 3, 1, 2)])
def test_two_pass_model_equals_oracle(shape):
    """Random residues and the all-(q-1) worst case; D0 = 600 spans three groups
    (the last one ragged)."""
    B, D0, D1, L, T = shape
    primes = PRIMES[:L]
    ct = synth.uniform_residues(71 + D0, synth.TAG_CT, (B, D0, 2, L, T), primes, limb_axis=3)
    db = synth.uniform_residues(72 + D0, synth.TAG_DB, (D0, D1, L, T), primes, limb_axis=2)
    assert np.array_equal(tc_model_rowsel_two_pass(ct, db, primes), oracle.rowsel(ct, db, primes))
    qm = np.array(primes, dtype=np.uint32)
    ct_w = np.broadcast_to(qm[None, None, None, :, None] - 1, ct.shape).copy()
    db_w = np.broadcast_to(qm[None, None, :, None] - 1, db.shape).copy()
    assert np.array_equal(tc_model_rowsel_two_pass(ct_w, db_w, primes), oracle.rowsel(ct_w, db_w, primes))


# ---- the INT8 (mma.sync) path: unsigned byte limbs, int32 diagonal sums ----

KFOLD = 8192                # rows per int32 accumulation in rowsel_imma.cu


def byte_limbs(x):
    x = np.asarray(x, dtype=np.int64)
    return np.stack([(x >> (8 * u)) & 0xFF for u in range(4)], axis=-1)


def test_imma_diagonal_bounds():
    """Per-row maxima of C_s = sum_{u+v=s} x_u y_v with bytes <= 255 and a top
    byte <= 15 (residues < 2^28): C_2 is the largest (3 * 255^2), so a fold
    interval of 8192 rows keeps every int32 accumulator below 2^31."""
    top = lambda u: 15 if u == 3 else 255
    maxima = [sum(top(u) * top(s - u) for u in range(4) if 0 <= s - u < 4) for s in range(7)]
    assert maxima == [65025, 130050, 195075, 137700, 72675, 7650, 225]
    assert max(maxima) == maxima[2]
    assert KFOLD * max(maxima) < 1 << 31 <= (KFOLD + 3000) * max(maxima)
    # the epilogue's sum over the seven diagonals, each < 2^31, times 2^(8s) mod q < 2^28
    assert 7 * (1 << 31) * (1 << 28) < 1 << 62


def imma_model_rowsel(ct, db, primes, kfold=KFOLD):
    """Byte limbs, seven diagonal int32 accumulators folded every `kfold` rows,
    folded sums reduced as sum_s A_s (2^(8s) mod q)."""
    ct = np.asarray(ct)
    db = np.asarray(db)
    B, D0, _, L, T = ct.shape
    D1 = db.shape[1]
    out = np.zeros((B, D1, 2, L, T), dtype=np.uint64)
    for l, q in enumerate(primes):
        q = int(q)
        c = [pow(2, 8 * s, q) for s in range(7)]
        for t in range(T):
            a = byte_limbs(ct[:, :, :, l, t].transpose(0, 2, 1).reshape(2 * B, D0))
            b = byte_limbs(db[:, :, l, t])
            res = np.zeros((2 * B, D1), dtype=object)
            for k0 in range(0, D0, kfold):
                k1 = min(D0, k0 + kfold)
                A = [sum(a[:, k0:k1, u] @ b[k0:k1, :, s - u] for u in range(4) if 0 <= s - u < 4) for s in range(7)]
                for s in range(7):
                    assert A[s].max() < 1 << 31
                res = (res + sum(A[s].astype(object) * c[s] for s in range(7)) % q) % q
            out[:, :, :, l, t] = res.astype(np.uint64).reshape(B, 2, D1).transpose(0, 2, 1)
    return out.astype(np.uint32)


@pytest.mark.parametrize("shape", [(2, 300, 4, 2, 2), (1, 70, 3, 1, 3)])
def test_imma_model_equals_oracle(shape):
    """Random residues, all q - 1, and residues whose three low bytes are all 255
    (0x0EFFFFFF, the C_2 extreme, below both primes), with a small fold interval
    so that several folds occur."""
    B, D0, D1, L, T = shape
    primes = PRIMES[:L]
    ct = synth.uniform_residues(81 + D0, synth.TAG_CT, (B, D0, 2, L, T), primes, limb_axis=3)
    db = synth.uniform_residues(82 + D0, synth.TAG_DB, (D0, D1, L, T), primes, limb_axis=2)
    assert np.array_equal(imma_model_rowsel(ct, db, primes, kfold=64), oracle.rowsel(ct, db, primes))
    for val in (None, 0x0EFFFFFF):
        qm = np.array(primes, dtype=np.uint32)
        fill_ct = qm[None, None, None, :, None] - 1 if val is None else np.uint32(val)
        fill_db = qm[None, None, :, None] - 1 if val is None else np.uint32(val)
        ct_w = np.broadcast_to(fill_ct, ct.shape).astype(np.uint32).copy()
        db_w = np.broadcast_to(fill_db, db.shape).astype(np.uint32).copy()
        assert np.all(ct_w < qm[None, None, None, :, None])
        assert np.array_equal(imma_model_rowsel(ct_w, db_w, primes), oracle.rowsel(ct_w, db_w, primes))


# ---- the CUDA-core path: 64-bit sums, one Barrett reduction every 256 rows ----

def test_cuda_core_accumulator_bound():
    """A reduced residue (< q) plus 256 products of residues below q < 2^28 fits in
    an unsigned 64-bit accumulator; 257 products of the largest residues would not."""
    for q in list(PRIMES) + [(1 << 28) - 1]:
        assert (q - 1) + 256 * (q - 1) ** 2 < 1 << 64
    assert 257 * ((1 << 28) - 2) ** 2 >= 1 << 64


def cc_model_rowsel(ct, db, primes, period=256):
    """uint64 multiply-accumulate, reduced mod q every `period` rows and at the end."""
    ct = np.asarray(ct, dtype=np.uint64)
    db = np.asarray(db, dtype=np.uint64)
    B, D0, _, L, T = ct.shape
    out = np.zeros((B, db.shape[1], 2, L, T), dtype=np.uint64)
    for l, q in enumerate(primes):
        qq = np.uint64(q)
        acc = np.zeros((B, db.shape[1], 2, T), dtype=np.uint64)
        for k0 in range(0, D0, period):
            for k in range(k0, min(D0, k0 + period)):
                acc += ct[:, k, :, l, :][:, None, :, :] * db[k, :, l, :][None, :, None, :]
            acc %= qq
        out[:, :, :, l, :] = acc
    return out.astype(np.uint32)


def test_cuda_core_model_equals_oracle():
    """All residues q - 1 over 600 rows (three reduction periods, the last ragged)
    and random residues: the uint64 schedule equals the oracle."""
    B, D0, D1, L, T = 2, 600, 3, 2, 3
    primes = PRIMES
    ct = synth.uniform_residues(91, synth.TAG_CT, (B, D0, 2, L, T), primes, limb_axis=3)
    db = synth.uniform_residues(92, synth.TAG_DB, (D0, D1, L, T), primes, limb_axis=2)
    assert np.array_equal(cc_model_rowsel(ct, db, primes), oracle.rowsel(ct, db, primes))
    qm = np.array(primes, dtype=np.uint32)
    ct_w = np.broadcast_to(qm[None, None, None, :, None] - 1, ct.shape).copy()
    db_w = np.broadcast_to(qm[None, None, :, None] - 1, db.shape).copy()
    assert np.array_equal(cc_model_rowsel(ct_w, db_w, primes), oracle.rowsel(ct_w, db_w, primes))


# ---------------------------------------------------------------------------
# The tensor-memory kernel's arithmetic: 12 digit products per modular MAC.
#
# Both operands are first centred: x -> x - q when x > (q-1)/2, congruent mod
# q and of magnitude below 2^27, so the product mod q is unchanged. Then
#   - ciphertext residues: y = x~ + O_A, O_A = 64 (1 + 2^7 + 2^14 + 2^21),
#     carried through the digit ring as z, the four 7-bit fields of y spread
#     one per byte (byte u = (y >> 7u) & 127 with bit 7 clear, byte 3 =
#     y >> 21 <= 128); digit d_u = field_u - 64 in [-64, 64];
#   - database residues: Y = v~ + O_B, O_B = 512 (1 + 2^10), digits
#     e_0 = (Y & 1023) - 512, e_1 = ((Y >> 10) & 1023) - 512, e_2 = Y >> 20
#     (arithmetic shift), e_v in [-512, 511] x [-128, 128];
#   - |d_u e_v| <= 2^15, so a group of 512 rows sums to at most 2^24: exact in
#     the fp32 accumulator; 12 group sums D_uv per output, recombined as
#     sum_uv D_uv (2^(7u + 10v) mod q) in 64 bits (< 2^55.6 per group), four
#     groups added (< 2^57.6) before one Barrett reduction of sum + off58.
# The fp16 digit of a byte is built as (0x6400 | field) - 1088 in fp16, which
# is exactly field - 64; the model does that in numpy float16.
# ---------------------------------------------------------------------------

O_A = 64 * (1 + (1 << 7) + (1 << 14) + (1 << 21))
O_B = 512 * (1 + (1 << 10))
GROUP12 = 512
FLUSH12 = 4


def ct_fields(x, q):
    """The ring encoding z of ciphertext residues x (uint32 array), bit for bit
    as the kernel computes it: y = centred(x) + O_A, a = y + 3 (y & ~0x3FFF)
    (bits 14.. up by 2), z = a + (a & 0x7F807F80) (bits 7..13 and 21.. of each
    16-bit half up by 1), in 32-bit arithmetic."""
    x = np.asarray(x, dtype=np.uint32)
    h = np.uint32((q - 1) // 2)
    y = (x + np.uint32(O_A) - np.where(x > h, np.uint32(q), np.uint32(0))).astype(np.uint32)
    a = (y + np.uint32(3) * (y & np.uint32(0xFFFFC000))).astype(np.uint32)
    return (a + (a & np.uint32(0x7F807F80))).astype(np.uint32)


def test_ring_encoding_is_the_field_split():
    """The add-based spreads give byte u = field u of y (7 bits, u < 3) and
    byte 3 = y >> 21, as the shift-and-mask definition does, for every residue
    of each prime's edge cases and a random sample."""
    rng = np.random.default_rng(23)
    for q in list(PRIMES) + [17, 97, 268042241]:
        h = (q - 1) // 2
        x = np.concatenate([rng.integers(0, q, 50000), [0, 1, h, h + 1, q - 1, q - 2]]).astype(np.int64)
        x = x[x < q]
        y = x + O_A - np.where(x > h, q, 0)
        assert y.min() >= 0 and y.max() < (1 << 29)
        want = (y & 0x7F) | (((y >> 7) & 0x7F) << 8) | (((y >> 14) & 0x7F) << 16) | ((y >> 21) << 24)
        assert np.array_equal(ct_fields(x.astype(np.uint32), q).astype(np.int64), want)


def ct_digit_fp16(z, u):
    """Digit u of ring words z as the kernel builds it: byte u as it is under
    0x6400 as an fp16, then one fp16 addition of -1088."""
    bits = ((z >> np.uint32(8 * u)) & np.uint32(0xFF)).astype(np.uint16) | np.uint16(0x6400)
    return (bits.view(np.float16) + np.float16(-1088.0)).astype(np.float16)


def db_digits12(v, q):
    """[..., 3] digits e_v of database residues (int64)."""
    v = np.asarray(v, dtype=np.int64)
    vt = np.where(v > (q - 1) // 2, v - q, v)
    Y = vt + O_B
    return np.stack([(Y & 1023) - 512, ((Y >> 10) & 1023) - 512, Y >> 20], axis=-1)


def tmem_model_rowsel(ct, db, primes, group=GROUP12, flush=FLUSH12, check_bounds=True):
    ct = np.asarray(ct)
    db = np.asarray(db)
    B, D0, _, L, T = ct.shape
    D1 = db.shape[1]
    out = np.zeros((B, D1, 2, L, T), dtype=np.uint32)
    for l, q in enumerate(primes):
        q = int(q)
        w = np.array([[pow(2, 7 * u + 10 * v, q) for v in range(3)] for u in range(4)], dtype=np.int64)
        off58 = -(-(1 << 58) // q) * q
        for t in range(T):
            z = ct_fields(ct[:, :, :, l, t].transpose(0, 2, 1).reshape(2 * B, D0), q)      # [2B][D0]
            a = [ct_digit_fp16(z, u).astype(np.float32) for u in range(4)]
            e = db_digits12(db[:, :, l, t], q).astype(np.float32)                             # [D0][D1][3]
            res = np.zeros((2 * B, D1), dtype=np.int64)
            acc = np.zeros((2 * B, D1), dtype=np.int64)
            groups = 0
            for g0 in range(0, D0, group):
                g1 = min(D0, g0 + group)
                for u in range(4):
                    for v in range(3):
                        D = a[u][:, g0:g1] @ e[g0:g1, :, v]                      # fp32 products and sums
                        if check_bounds:
                            assert np.all(np.abs(D) <= 2 ** 24)
                        acc += D.astype(np.int64) * w[u, v]
                groups += 1
                if groups == flush or g1 == D0:
                    if check_bounds:
                        assert np.all(np.abs(acc) < 2 ** 58)
                    res = (res + (acc + off58) % q) % q
                    acc[:] = 0
                    groups = 0
            out[:, :, :, l, t] = res.reshape(B, 2, D1).transpose(0, 2, 1).astype(np.uint32)
    return out


def test_ring_encoding_and_fp16_digits_reconstruct_the_centred_residue():
    rng = np.random.default_rng(17)
    for q in list(PRIMES) + [17, 97, 268042241]:
        h = (q - 1) // 2
        x = np.concatenate([rng.integers(0, q, 4000), [0, 1, h, h + 1, q - 1, q - 1056832, q - 2]]).astype(np.uint32)
        x = x[x < q]
        z = ct_fields(x, q)
        d = np.stack([ct_digit_fp16(z, u).astype(np.int64) for u in range(4)], axis=-1)
        assert d.min() >= -64 and d.max() <= 64
        xt = np.where(x.astype(np.int64) > h, x.astype(np.int64) - q, x.astype(np.int64))
        assert np.array_equal((d * np.array([1, 1 << 7, 1 << 14, 1 << 21])).sum(-1), xt)
        e = db_digits12(x, q)
        assert e[..., :2].min() >= -512 and e[..., :2].max() <= 511 and np.abs(e[..., 2]).max() <= 128
        assert np.array_equal((e * np.array([1, 1 << 10, 1 << 20])).sum(-1), xt)
    # every byte and its fp16 image exact: the fp16 arithmetic equals the integer one
    z = np.arange(0, 1 << 16, dtype=np.uint32) * np.uint32(0x01010101 // 257 + 1)
    for u in range(4):
        f = (z >> np.uint32(8 * u)) & np.uint32(0xFF)
        assert np.array_equal(ct_digit_fp16(z, u).astype(np.int64), f.astype(np.int64) - 64)


def test_ring_encoding_clears_bit_7_of_the_low_fields():
    """The converters take each byte of a ring word as it is, so the encoding
    must leave bit 7 of bytes 0..2 clear for every residue below q."""
    rng = np.random.default_rng(19)
    for q in list(PRIMES) + [17, 268042241]:
        h = (q - 1) // 2
        x = np.concatenate([rng.integers(0, q, 20000), [0, h, h + 1, q - 1]]).astype(np.uint32)
        z = ct_fields(x, q)
        for u in range(3):
            assert ((z >> np.uint32(8 * u + 7)) & np.uint32(1)).max() == 0


def test_tmem_model_matches_oracle_random():
    primes = PRIMES
    B, D0, D1, L, T = 3, 1100, 9, 2, 2          # three groups, the last one ragged
    ct = synth.ct_tensor(301, B, D0, L, T, primes)
    db = synth.db_tensor(301, D0, D1, L, T, primes)
    assert np.array_equal(tmem_model_rowsel(ct, db, primes), oracle.rowsel(ct, db, primes))


def test_tmem_model_extreme_digits_reach_the_bound():
    """Residues whose digits sit at the ends of their ranges: ciphertext
    q - 1056832 (centred -1056832: digits -64, -64, -64, 0) against database
    q - 524800 (centred -524800: digits -512, -512, 0), so the group sums of
    the (u < 3, v < 2) pairs reach exactly 2^24; and the top ciphertext digit at
    +64 against -512. The model stays exact and equals D0 * x * y mod q."""
    primes = PRIMES
    B, D0, D1, L, T = 1, 2048, 2, 2, 1
    for (xs, ys) in [((lambda q: q - 1056832), (lambda q: q - 524800)),
                     ((lambda q: 133160896 + 7), (lambda q: q - 524800)),
                     ((lambda q: (q - 1) // 2), (lambda q: (q + 1) // 2))]:
        ct = np.empty((B, D0, 2, L, T), dtype=np.uint32)
        db = np.empty((D0, D1, L, T), dtype=np.uint32)
        for l, q in enumerate(primes):
            ct[:, :, :, l] = xs(q)
            db[:, :, l] = ys(q)
        got = tmem_model_rowsel(ct, db, primes)
        for l, q in enumerate(primes):
            assert np.all(got[:, :, :, l] == (D0 * xs(q) * ys(q)) % q)
    q = primes[0]
    z = ct_fields(np.array([q - 1056832], dtype=np.uint32), q)
    assert [int(ct_digit_fp16(z, u)[0]) for u in range(4)] == [-64, -64, -64, 0]
    assert db_digits12(np.array([q - 524800]), q).tolist() == [[-512, -512, 0]]
    z = ct_fields(np.array([133160896 + 7], dtype=np.uint32), q)
    assert int(ct_digit_fp16(z, 3)[0]) == 64


def test_tmem_model_negative_control_group_too_long():
    """With 1025-row groups a partial sum passes 2^24 and fp32 rounds it: the
    model (bounds unchecked) then differs from the oracle, so the 512-row
    limit is what keeps the arithmetic exact."""
    primes = PRIMES[:1]
    q = primes[0]
    B, D0, D1, L, T = 1, 1025, 1, 1, 1
    ct = np.full((B, D0, 2, L, T), q - 1056832, dtype=np.uint32)
    db = np.full((D0, D1, L, T), q - 524800, dtype=np.uint32)
    ct[:, -1] = 1          # one more product of 1 after the sums reached 2^24 + ...
    db[-1] = 1
    want = oracle.rowsel(ct, db, primes)
    assert np.array_equal(tmem_model_rowsel(ct, db, primes), want)            # 512-row groups: exact
    bad = tmem_model_rowsel(ct, db, primes, group=1025, check_bounds=False)
    assert not np.array_equal(bad, want)
