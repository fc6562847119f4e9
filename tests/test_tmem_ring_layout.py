"""CPU model of the tensor-memory kernel's ring tile layout (rowsel_tmem.cu):
the ingest's byte transpose of encoded residues into digit planes, the
swizzled 16-byte chunk positions, and the converters' per-digit reads.

The ingest lane (k octet j, row parity, slot half) takes the slots of its half
one at a time and holds the ring words of its octet in position order, position
kk carrying k offset kk ^ (j & 1) (the order that spreads its 4-byte box reads
over 8 banks). It transposes them with byte permutations into four digit
planes, k in order, and stores chunk 2j (digits 0, 1) and chunk 2j + 1 (digits
2, 3) of its row m at positions c16 ^ (m % 8).
A converter thread (row m, digit u) reads 8 bytes per octet and builds fp16
pairs (0x6400 | byte) - 1088. Checked: every converter read returns byte u of
the row's words in k order, the fp16 pairs equal field - 64, the warp's reads
are bank-conflict-free, the ingest's box reads cover the box once with 4 lanes
per bank, and leaving out the swap of odd octets is caught.
"""

import numpy as np
import pytest


def byte_perm(a, b, s):
    """PRMT in its default mode: result byte n = byte (s >> 4n) & 7 of the
    8-byte value b:a (selector nibbles below 8, no sign replication)."""
    src = (int(b) << 32) | int(a)
    r = 0
    for n in range(4):
        k = (s >> (4 * n)) & 0xF
        assert k < 8
        r |= ((src >> (8 * k)) & 0xFF) << (8 * n)
    return r


def digit_planes(w, sa, sb):
    t0, t1 = byte_perm(w[0], w[1], sa), byte_perm(w[0], w[1], sb)
    t2, t3 = byte_perm(w[2], w[3], sa), byte_perm(w[2], w[3], sb)
    return [byte_perm(t0, t2, 0x5410), byte_perm(t0, t2, 0x7632), byte_perm(t1, t3, 0x5410),
            byte_perm(t1, t3, 0x7632)]


def ingest_tile(zrows, swap_fix=True):
    """zrows: [32][64] ring words of one slot and k-chunk -> the 8 KB tile as
    [32 rows][16 chunks][4 words]."""
    tile = np.zeros((32, 16, 4), dtype=np.uint64)
    for m in range(32):
        for j in range(8):
            j0 = j & 1
            w = [int(zrows[m][8 * j + (kk ^ j0)]) for kk in range(8)]   # position order
            if swap_fix and j0:
                sa, sb = 0x1504, 0x3726
            else:
                sa, sb = 0x5140, 0x7362
            pl, ph = digit_planes(w[:4], sa, sb), digit_planes(w[4:], sa, sb)
            tile[m, (2 * j) ^ (m & 7)] = [pl[0], ph[0], pl[1], ph[1]]
            tile[m, (2 * j + 1) ^ (m & 7)] = [pl[2], ph[2], pl[3], ph[3]]
    return tile


def converter_read(tile, m, u, j):
    """The uint2 a converter thread (row m, digit u) reads for octet j."""
    c = (2 * j + (u >> 1)) ^ (m & 7)
    return int(tile[m, c, 2 * (u & 1)]), int(tile[m, c, 2 * (u & 1) + 1])


def plane_pair_fp16(w, sel):
    t = byte_perm(w, 0x64646464, sel)
    h = np.array([t & 0xFFFF, t >> 16], dtype=np.uint16).view(np.float16)
    return (h + np.float16(-1088.0)).astype(np.float16)


def random_ring_words(rng, n):
    """Ring words with the encoding's shape: bytes 0..2 of 7 bits, byte 3 up to 128."""
    f = rng.integers(0, 128, size=(n, 4), dtype=np.uint64)
    f[:, 3] = rng.integers(0, 129, size=n, dtype=np.uint64)
    return f[:, 0] | (f[:, 1] << 8) | (f[:, 2] << 16) | (f[:, 3] << 24)


def test_converter_reads_digit_planes_in_k_order():
    rng = np.random.default_rng(5)
    z = random_ring_words(rng, 32 * 64).reshape(32, 64)
    tile = ingest_tile(z)
    for m in range(32):
        for u in range(4):
            for j in range(8):
                lo, hi = converter_read(tile, m, u, j)
                got = [(lo >> (8 * b)) & 0xFF for b in range(4)] + [(hi >> (8 * b)) & 0xFF for b in range(4)]
                want = [(int(z[m][8 * j + k]) >> (8 * u)) & 0xFF for k in range(8)]
                assert got == want, (m, u, j)
                # fp16 pairs (k, k + 1) as the converter builds them: field - 64
                vals = np.concatenate([plane_pair_fp16(lo, 0x5140), plane_pair_fp16(lo, 0x5342),
                                       plane_pair_fp16(hi, 0x5140), plane_pair_fp16(hi, 0x5342)])
                assert np.array_equal(vals.astype(np.int64), np.array(want, dtype=np.int64) - 64)


def test_every_tile_word_is_written_once():
    z = np.arange(32 * 64, dtype=np.uint64).reshape(32, 64) * 0x01010101 % (1 << 31)
    tile = ingest_tile(z)
    # each (row, chunk) position written exactly once: the positions of a row
    # are a permutation of its 16 chunks
    for m in range(32):
        pos = sorted(((2 * j + h) ^ (m & 7)) for j in range(8) for h in range(2))
        assert pos == list(range(16))


def test_converter_reads_are_bank_conflict_free():
    """A converter warp (quarter qw) is lanes u = lane >> 3, m_lo = lane & 7 on
    rows qw * 8 + m_lo; one 8-byte read per lane per octet: 256 bytes, so two
    wavefronts at best, i.e. every 4-byte bank touched exactly twice."""
    row_bytes = 256
    for qw in range(4):
        for j in range(8):
            banks = np.zeros(32, dtype=int)
            for lane in range(32):
                u, m = lane >> 3, qw * 8 + (lane & 7)
                c = (2 * j + (u >> 1)) ^ (m & 7)
                addr = m * row_bytes + c * 16 + (u & 1) * 8
                for w in range(2):
                    banks[(addr // 4 + w) % 32] += 1
            assert banks.max() == 2 and banks.min() == 2, (qw, j, banks)


def test_missing_odd_octet_swap_is_caught():
    """Sensitivity: transposing odd octets with the in-order selectors (their
    words sit pairwise swapped) gives converters wrong k order."""
    rng = np.random.default_rng(6)
    z = random_ring_words(rng, 32 * 64).reshape(32, 64)
    tile = ingest_tile(z, swap_fix=False)
    bad = 0
    for m in range(32):
        for u in range(4):
            lo, hi = converter_read(tile, m, u, 1)
            got = [(lo >> (8 * b)) & 0xFF for b in range(4)] + [(hi >> (8 * b)) & 0xFF for b in range(4)]
            want = [(int(z[m][8 + k]) >> (8 * u)) & 0xFF for k in range(8)]
            bad += got != want
    assert bad > 0


@pytest.mark.parametrize("u", [0, 1, 2, 3])
def test_plane_bytes_need_no_mask(u):
    """Bytes 0..2 of a ring word have bit 7 clear (the encoding leaves a zero
    bit above each 7-bit field), so 0x6400 | byte is field + 1024 exactly."""
    import tests.test_tc_arithmetic as ta
    rng = np.random.default_rng(7)
    for q in ta.PRIMES:
        x = rng.integers(0, q, 20000).astype(np.uint32)
        z = ta.ct_fields(x, q)
        b = (z >> np.uint32(8 * u)) & np.uint32(0xFF)
        assert b.max() <= (127 if u < 3 else 128)


def box_word(cb, j, kk, rp, sh, i):
    """Index of the 4-byte box word an ingest thread reads: client cb of the
    box, k octet j, position kk (k offset kk ^ (j & 1)), row parity rp, slot
    half sh, slot i of the half. Box layout [client][k][row parity][8 slots]."""
    return (((cb * 64 + j * 8 + (kk ^ (j & 1))) * 2 + rp) * 2 + sh) * 4 + i


def ingest_lane(lane):
    j, rp = lane >> 2, (lane >> 1) & 1
    sh = (lane & 1) ^ ((j >> 1) & 1)
    return j, rp, sh


def test_ingest_box_reads_cover_the_box_once():
    """The 8 warps (one client each) read every word of an 8-client box exactly
    once: k = 8 j + (kk ^ (j & 1)) runs over 0..63 for each octet."""
    seen = np.zeros(8 * 64 * 2 * 8, dtype=int)
    for cb in range(8):
        for lane in range(32):
            j, rp, sh = ingest_lane(lane)
            for i in range(4):
                for kk in range(8):
                    seen[box_word(cb, j, kk, rp, sh, i)] += 1
    assert seen.min() == 1 and seen.max() == 1


@pytest.mark.parametrize("swaps", [True, False])
def test_ingest_box_read_bank_spread(swaps):
    """Each 4-byte read instruction (fixed kk and i) of a warp touches 8 banks
    with 4 lanes each; without the k-offset and slot-half swaps it would touch
    4 banks with 8 lanes each."""
    for kk in range(8):
        for i in range(4):
            banks = np.zeros(32, dtype=int)
            for lane in range(32):
                j, rp, sh = ingest_lane(lane)
                if not swaps:
                    sh = lane & 1
                    w = (((0 * 64 + j * 8 + kk) * 2 + rp) * 2 + sh) * 4 + i
                else:
                    w = box_word(0, j, kk, rp, sh, i)
                banks[w % 32] += 1
            used = banks[banks > 0]
            if swaps:
                assert len(used) == 8 and used.max() == 4, (kk, i, banks)
            else:
                assert len(used) == 4 and used.max() == 8, (kk, i, banks)
