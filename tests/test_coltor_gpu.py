"""GPU ColTor vs the CPU oracle, bit-exact (modular integer work: tolerance 0),
plus decryption checks of the tournament at full ring size. The library picks
one of two stage kernels per stage by node count (a cluster per node split by
limb, or by polynomial and limb when the nodes are few); the shapes below
reach both.

All calls go through the C ABI (libgpir.so) via the ctypes binding."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

P28 = synth.PRIMES_28


@pytest.fixture(scope="module")
def g():
    from tests import gpu_util
    return gpu_util.lib()


def _gpu_coltor(g, primes, N, ct, rgsw):
    """ct [B][D1][2][L][N], rgsw [B][stages][2 ell][2][L][N] (numpy) -> [B][2][L][N]."""
    import torch
    from tests.gpu_util import to_dev, to_host
    B, D1 = ct.shape[0], ct.shape[1]
    params = g.gpir_params_create(N, list(primes))
    try:
        out = torch.full((B, 2, len(primes), N), -1, dtype=torch.int32, device="cuda")
        g.gpir_coltor(params, B, D1, to_dev(ct), to_dev(rgsw), out)
        torch.cuda.synchronize()
        g.gpir_sync(None, 20000)
        return to_host(out)
    finally:
        g.gpir_params_destroy(params)


SHAPES = [
    # (B, D1, L, N)            what it covers
    (1, 2, 2, 16),             # one node, smallest ring with the 28-bit primes' 3 digits
    (2, 4, 2, 64),             # two stages, two clients
    (3, 8, 1, 32),             # one limb: 2 digits, no CRT
    (1, 16, 2, 512),           # four stages (ping-pong workspace), N = one CTA's width
    (2, 2, 2, 1024),           # points per thread > 1
    (1, 2, 2, 4096),           # the workload ring size
    (10, 64, 2, 32),           # >= 2 CTAs per SM of nodes: the limb kernel in the early stages, the split one late
    (10, 64, 1, 32),           # the same with one limb
    (2, 4, 1, 256),            # logn = 8: a radix-4 middle round
    (1, 4, 2, 2048),           # logn = 11: radix-8 + radix-4 middle rounds
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "B%d_D1%d_L%d_N%d" % s)
def test_coltor_vs_oracle_random(g, shape):
    """Uniform random ciphertexts and RGSW rows: every output residue equal."""
    B, D1, L, N = shape
    primes = P28[:L]
    ell = oracle.gadget_digits(primes)
    stages = D1.bit_length() - 1
    ct = synth.uniform_residues(500 + N + D1, synth.TAG_COLTOR, (B, D1, 2, L, N), primes, limb_axis=3)
    rgsw = synth.uniform_residues(600 + N + D1, synth.TAG_RGSW, (B, stages, 2 * ell, 2, L, N), primes, limb_axis=4)
    got = _gpu_coltor(g, primes, N, ct, rgsw)
    for c in range(B):
        want = oracle.coltor(ct[c], rgsw[c], primes)
        assert np.array_equal(got[c], want), "client %d: %d of %d residues differ" % (
            c, int((got[c] != want).sum()), want.size)


def test_gadget_digits_match_oracle(g):
    for primes in (P28[:1], P28):
        params = g.gpir_params_create(64, list(primes))
        try:
            assert g.gpir_coltor_gadget_digits(params) == oracle.gadget_digits(primes)
        finally:
            g.gpir_params_destroy(params)


@pytest.mark.parametrize("L", [1, 2])
def test_coltor_toy_decrypts_to_record_full_ring(g, L):
    """N = 4096, D1 = 64 (the 32-client workload's column count): the GPU result
    of a noiseless toy tournament decrypts to the selected record, for several
    column indices in one batch."""
    N, D1 = 4096, 64
    primes = P28[:L]
    ell = oracle.gadget_digits(primes)
    jstars = [0, 37, 63]
    cts, rgsws, secrets, recs = [], [], [], []
    for c, js in enumerate(jstars):
        ct, rgsw, s, rec = synth.toy_coltor_inputs(700 + c, D1, L, N, primes, js, ell)
        cts.append(ct)
        rgsws.append(rgsw)
        secrets.append(s)
        recs.append(rec)
    got = _gpu_coltor(g, primes, N, np.stack(cts), np.stack(rgsws))
    for c, js in enumerate(jstars):
        for l, q in enumerate(primes):
            a = got[c, 0, l].astype(np.uint64)
            b = got[c, 1, l].astype(np.uint64)
            m = (b + np.uint64(q) - (a * secrets[c][l].astype(np.uint64)) % np.uint64(q)) % np.uint64(q)
            assert np.array_equal(m, recs[c][js][l].astype(np.uint64)), "client %d limb %d" % (c, l)


def test_rowsel_then_coltor_returns_db_entry(g):
    """Tensor-core RowSel with toy one-hot queries, then ColTor on its outputs,
    all on the GPU at N = 4096: each client decrypts DB[i*][j*]."""
    import torch
    from tests.gpu_util import DbHandle, to_dev, to_host
    N, L, D0, D1 = 4096, 2, 64, 16
    primes = P28
    ell = oracle.gadget_digits(primes)
    db = synth.uniform_residues(801, synth.TAG_DB, (D0, D1, L, N), primes, limb_axis=2)
    picks = [(3, 5), (60, 15), (0, 0)]
    h = DbHandle(g, db, N, primes, path_mask=4)
    try:
        cts, secrets, rgsws = [], [], []
        for c, (i, j) in enumerate(picks):
            ct, s = synth.toy_rlwe_selection(810 + c, D0, L, N, primes, i)
            cts.append(ct)
            secrets.append(s)
            rgsws.append(np.stack([synth.toy_rgsw(810 + c, st, (j >> st) & 1, s, L, N, primes, ell)
                                   for st in range(D1.bit_length() - 1)]))
        B = len(picks)
        rows = h.rowsel(to_dev(np.stack(cts)), B, 4)            # [B][D1][2][L][N] on the device
        out = torch.full((B, 2, L, N), -1, dtype=torch.int32, device="cuda")
        g.gpir_coltor(h.params, B, D1, rows, to_dev(np.stack(rgsws)), out)
        torch.cuda.synchronize()
        g.gpir_sync(None, 20000)
        got = to_host(out)
    finally:
        h.close()
    for c, (i, j) in enumerate(picks):
        for l, q in enumerate(primes):
            a = got[c, 0, l].astype(np.uint64)
            b = got[c, 1, l].astype(np.uint64)
            m = (b + np.uint64(q) - (a * secrets[c][l].astype(np.uint64)) % np.uint64(q)) % np.uint64(q)
            assert np.array_equal(m, db[i, j, l].astype(np.uint64)), "client %d limb %d" % (c, l)


def test_coltor_argument_errors(g):
    import torch
    params = g.gpir_params_create(64, list(P28))
    try:
        buf = torch.zeros(1 << 16, dtype=torch.int32, device="cuda")
        for d1 in (0, 1, 3, 6):
            assert g.lib.gpir_coltor(params, 1, d1, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), None) == \
                g.GPIR_EINVAL
        assert g.lib.gpir_coltor(params, 0, 4, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), None) == \
            g.GPIR_EINVAL
    finally:
        g.gpir_params_destroy(params)
    p3 = g.gpir_params_create(64, [268369921, 268361729, 268271617])
    try:
        buf = torch.zeros(16, dtype=torch.int32, device="cuda")
        assert g.lib.gpir_coltor(p3, 1, 2, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), None) == g.GPIR_ENOTSUP
    finally:
        g.gpir_params_destroy(p3)


def test_coltor_bench_configuration_decrypts(g):
    """The bench's ColTor configuration exactly (32 clients x 64 ciphertexts,
    N = 4096, 2 limbs: limb kernel for stages 0-3, split kernel for 4-5), with
    noiseless toy inputs: every client decrypts to its selected record."""
    N, L, D1, B = 4096, 2, 64, 32
    primes = P28
    ell = oracle.gadget_digits(primes)
    cts, rgsws, secrets, recs, picks = [], [], [], [], []
    for c in range(B):
        js = (c * 37 + 5) % D1
        ct, rgsw, s, rec = synth.toy_coltor_inputs(1000 + c, D1, L, N, primes, js, ell)
        cts.append(ct)
        rgsws.append(rgsw)
        secrets.append(s)
        recs.append(rec)
        picks.append(js)
    got = _gpu_coltor(g, primes, N, np.stack(cts), np.stack(rgsws))
    for c in range(B):
        for l, q in enumerate(primes):
            a = got[c, 0, l].astype(np.uint64)
            b = got[c, 1, l].astype(np.uint64)
            m = (b + np.uint64(q) - (a * secrets[c][l].astype(np.uint64)) % np.uint64(q)) % np.uint64(q)
            assert np.array_equal(m, recs[c][picks[c]][l].astype(np.uint64)), "client %d limb %d" % (c, l)


def test_coltor_zero_inputs_give_zero(g):
    """All-zero ciphertexts (and RGSW rows) give an all-zero result; all-zero
    differences with random RGSW rows give back ct_0 exactly."""
    primes = P28
    B, D1, L, N = 2, 8, 2, 256
    ell = oracle.gadget_digits(primes)
    ct = np.zeros((B, D1, 2, L, N), dtype=np.uint32)
    rgsw = synth.uniform_residues(951, synth.TAG_RGSW, (B, 3, 2 * ell, 2, L, N), primes, limb_axis=4)
    assert not _gpu_coltor(g, primes, N, ct, np.zeros_like(rgsw)).any()
    same = synth.uniform_residues(952, synth.TAG_COLTOR, (B, 1, 2, L, N), primes, limb_axis=3)
    ct = np.repeat(same, D1, axis=1)                     # every pair differs by zero
    got = _gpu_coltor(g, primes, N, ct, rgsw)
    assert np.array_equal(got, same[:, 0])
