"""GPU ExpandQuery vs the CPU oracle, bit-exact (modular integer work: tolerance
0), plus decryption checks at full ring size and the three server phases
chained on the GPU. The library picks one of two stage kernels per stage by
node count (a cluster per node split by limb, or by limb and digit when the
nodes are few); the shapes below reach both.

All calls go through the C ABI (libgpir.so) via the ctypes binding."""

import numpy as np
import pytest

import oracle
import synth
from tests import expand_util as eu

pytestmark = pytest.mark.gpu

P28 = synth.PRIMES_28


@pytest.fixture(scope="module")
def g():
    from tests import gpu_util
    return gpu_util.lib()


def _gpu_expand(g, primes, N, query, evk, n_out):
    """query [B][2][L][N], evk [B][J][ell][2][L][N] (numpy) -> [B][n_out][2][L][N]."""
    import torch
    from tests.gpu_util import to_dev, to_host
    B, J = query.shape[0], evk.shape[1]
    params = g.gpir_params_create(N, list(primes))
    try:
        out = torch.full((B, n_out, 2, len(primes), N), -1, dtype=torch.int32, device="cuda")
        g.gpir_expand_query(params, B, J, n_out, to_dev(query), to_dev(evk) if J else None, out)
        torch.cuda.synchronize()
        g.gpir_sync(None, 20000)
        return to_host(out)
    finally:
        g.gpir_params_destroy(params)


SHAPES = [
    # (B, J, n_out, L, N)       what it covers
    (1, 1, 2, 2, 16),           # one node, smallest ring
    (2, 2, 3, 2, 64),           # ragged n_out: the last stage writes one out1 of two
    (3, 3, 8, 1, 32),           # one limb, three stages
    (2, 4, 11, 2, 512),         # ragged n_out over four stages
    (1, 3, 5, 2, 128),          # logn = 7: a radix-2 middle round
    (1, 2, 4, 2, 4096),         # the workload ring size
    (20, 5, 32, 2, 32),         # >= 2 CTAs per SM of nodes in the last stage: the limb kernel there, the split one before
    (20, 5, 29, 1, 32),         # the same with one limb, ragged
    (1, 4, 16, 1, 256),         # logn = 8: a radix-4 middle round
    (2, 3, 8, 2, 1024),         # logn = 10: two radix-4 middle rounds
    (2, 3, 7, 2, 2048),         # logn = 11: radix-8 + radix-4 middle rounds
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "B%d_J%d_n%d_L%d_N%d" % s)
def test_expand_vs_oracle_random(g, shape):
    """Uniform random query and keys: every output residue equal."""
    B, J, n_out, L, N = shape
    primes = P28[:L]
    ell = oracle.gadget_digits(primes)
    query = synth.uniform_residues(900 + N + J, eu.TAG_QUERY, (B, 2, L, N), primes, limb_axis=2)
    evk = synth.uniform_residues(950 + N + J, eu.TAG_EVK, (B, J, ell, 2, L, N), primes, limb_axis=4)
    got = _gpu_expand(g, primes, N, query, evk, n_out)
    for c in range(B):
        want = oracle.expand_query(query[c], evk[c], primes, n_out)
        assert np.array_equal(got[c], want), "client %d: %d of %d residues differ" % (
            c, int((got[c] != want).sum()), want.size)


def test_expand_zero_stages_copies(g):
    primes = P28
    query = synth.uniform_residues(3, eu.TAG_QUERY, (2, 2, 2, 64), primes, limb_axis=2)
    got = _gpu_expand(g, primes, 64, query, np.zeros((2, 0, 3, 2, 2, 64), dtype=np.uint32), 1)
    assert np.array_equal(got[:, 0], query)


@pytest.mark.parametrize("L", [1, 2])
def test_expand_toy_decrypts_to_scaled_message_full_ring(g, L):
    """N = 4096, J = 8, 256 outputs (the 32-client workload's D0): a noiseless
    toy query whose message has coefficients only below 2^J expands into
    ciphertexts of the constants 2^J m_r, for two clients at once."""
    N, J = 4096, 8
    primes = P28[:L]
    ell = oracle.gadget_digits(primes)
    queries, evks, secrets, msgs = [], [], [], []
    for c in range(2):
        q_, evk, s, m = eu.toy_expand_inputs(40 + c, J, L, N, primes, ell)
        # keep only coefficients below 2^J: re-encrypt that message under the same key
        m = [x if i < (1 << J) else 0 for i, x in enumerate(m)]
        for l, q in enumerate(primes):
            M = oracle.ntt_negacyclic([x % q for x in m], q, oracle.psi_2n(q, N))
            q_[1, l] = ((q_[0, l].astype(np.uint64) * s[l].astype(np.uint64) + M) % np.uint64(q)).astype(np.uint32)
        queries.append(q_)
        evks.append(evk)
        secrets.append(s)
        msgs.append(m)
    got = _gpu_expand(g, primes, N, np.stack(queries), np.stack(evks), 1 << J)
    for c in range(2):
        for l, q in enumerate(primes):
            a = got[c, :, 0, l].astype(np.uint64)
            b = got[c, :, 1, l].astype(np.uint64)
            ph = (b + np.uint64(q) - (a * secrets[c][l].astype(np.uint64)[None, :]) % np.uint64(q)) % np.uint64(q)
            want = np.array([((1 << J) * msgs[c][r]) % q for r in range(1 << J)], dtype=np.uint64)
            assert np.array_equal(ph, np.repeat(want[:, None], N, axis=1)), "client %d limb %d" % (c, l)


def test_expand_bench_configuration_decrypts(g):
    """The bench's ExpandQuery configuration exactly (32 clients, J = 9 stages,
    ragged n_out = 274, N = 4096, 2 limbs), with noiseless toy inputs whose
    messages have coefficients below 2^J: output r of each client decrypts to
    the constant 2^J m_r."""
    N, L, J, n_out, B = 4096, 2, 9, 274, 32
    primes = P28
    ell = oracle.gadget_digits(primes)
    psis = [oracle.psi_2n(q, N) for q in primes]
    queries, evks, secrets, msgs = [], [], [], []
    for c in range(B):
        q_, evk, s, m = eu.toy_expand_inputs(2000 + c, J, L, N, primes, ell)
        m = [x if i < n_out else 0 for i, x in enumerate(m)]
        for l, q in enumerate(primes):
            M = oracle.ntt_negacyclic([x % q for x in m], q, psis[l])
            q_[1, l] = ((q_[0, l].astype(np.uint64) * s[l].astype(np.uint64) + M) % np.uint64(q)).astype(np.uint32)
        queries.append(q_)
        evks.append(evk)
        secrets.append(s)
        msgs.append(m)
    got = _gpu_expand(g, primes, N, np.stack(queries), np.stack(evks), n_out)
    for c in range(B):
        for l, q in enumerate(primes):
            a = got[c, :, 0, l].astype(np.uint64)
            b = got[c, :, 1, l].astype(np.uint64)
            ph = (b + np.uint64(q) - (a * secrets[c][l].astype(np.uint64)[None, :]) % np.uint64(q)) % np.uint64(q)
            want = np.array([((1 << J) * msgs[c][r]) % q for r in range(n_out)], dtype=np.uint64)
            assert np.array_equal(ph, np.repeat(want[:, None], N, axis=1)), "client %d limb %d" % (c, l)


def test_expand_rowsel_coltor_returns_scaled_db_entry(g):
    """The three server phases chained on the GPU at N = 4096: a toy query
    encrypting X^(i*) expands into a one-hot selection vector (scaled by 2^J),
    tensor-core RowSel selects row i*, ColTor (toy RGSW bits of j*) selects
    column j*; each client decrypts 2^J DB[i*][j*]."""
    import torch
    from tests.gpu_util import DbHandle, to_dev, to_host
    N, L, D0, D1 = 4096, 2, 64, 8
    J = 6
    primes = P28
    ell = oracle.gadget_digits(primes)
    db = synth.uniform_residues(811, synth.TAG_DB, (D0, D1, L, N), primes, limb_axis=2)
    picks = [(5, 3), (63, 0), (0, 7)]
    h = DbHandle(g, db, N, primes, path_mask=4)
    try:
        queries, evks, secrets, rgsws = [], [], [], []
        for c, (i, j) in enumerate(picks):
            q_, evk, s, _ = eu.toy_expand_inputs(820 + c, J, L, N, primes, ell)
            for l, q in enumerate(primes):
                M = oracle.monomial_ntt(i, q, N)
                q_[1, l] = ((q_[0, l].astype(np.uint64) * s[l].astype(np.uint64) + M) % np.uint64(q)).astype(np.uint32)
            queries.append(q_)
            evks.append(evk)
            secrets.append(s)
            rgsws.append(np.stack([synth.toy_rgsw(820 + c, st, (j >> st) & 1, s, L, N, primes, ell)
                                   for st in range(D1.bit_length() - 1)]))
        B = len(picks)
        sel = torch.full((B, D0, 2, L, N), -1, dtype=torch.int32, device="cuda")
        g.gpir_expand_query(h.params, B, J, D0, to_dev(np.stack(queries)), to_dev(np.stack(evks)), sel)
        rows = h.rowsel(sel, B, 4)                                   # [B][D1][2][L][N]
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
            want = (db[i, j, l].astype(np.uint64) * np.uint64(1 << J)) % np.uint64(q)
            assert np.array_equal(m, want), "client %d limb %d" % (c, l)


def test_expand_argument_errors(g):
    import torch
    params = g.gpir_params_create(64, list(P28))
    try:
        buf = torch.zeros(1 << 18, dtype=torch.int32, device="cuda")
        p = buf.data_ptr()
        call = g.lib.gpir_expand_query
        assert call(params, 1, 2, 5, p, p, p, None) == g.GPIR_EINVAL      # n_out > 2^J
        assert call(params, 1, 2, 0, p, p, p, None) == g.GPIR_EINVAL      # n_out = 0
        assert call(params, 0, 2, 4, p, p, p, None) == g.GPIR_EINVAL      # batch = 0
        assert call(params, 1, 7, 4, p, p, p, None) == g.GPIR_EINVAL      # J > log2 N
        assert call(params, 1, 2, 4, p, None, p, None) == g.GPIR_EINVAL   # no keys
    finally:
        g.gpir_params_destroy(params)
    for n, primes in [(64, [268369921, 268361729, 268271617]), (8, [268369921])]:
        p3 = g.gpir_params_create(n, primes)
        try:
            buf = torch.zeros(1 << 12, dtype=torch.int32, device="cuda")
            assert g.lib.gpir_expand_query(p3, 1, 1, 2, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), None) == \
                g.GPIR_ENOTSUP
        finally:
            g.gpir_params_destroy(p3)


def test_pir_batch_equals_the_three_calls_and_decrypts(g):
    """gpir_pir_batch (ExpandQuery -> RowSel -> ColTor in one call, caller-owned
    intermediate buffers) returns exactly what the three separate calls return,
    for every RowSel path, and decrypts to 2^J DB[i*][j*]."""
    import torch
    from tests.gpu_util import DbHandle, to_dev, to_host
    N, L, D0, D1, J = 1024, 2, 48, 4, 6
    primes = P28
    ell = oracle.gadget_digits(primes)
    db = synth.uniform_residues(911, synth.TAG_DB, (D0, D1, L, N), primes, limb_axis=2)
    picks = [(47, 1), (0, 3)]
    h = DbHandle(g, db, N, primes, path_mask=0)
    try:
        queries, evks, secrets, rgsws = [], [], [], []
        for c, (i, j) in enumerate(picks):
            q_, evk, s, _ = eu.toy_expand_inputs(920 + c, J, L, N, primes, ell)
            for l, q in enumerate(primes):
                M = oracle.monomial_ntt(i, q, N)
                q_[1, l] = ((q_[0, l].astype(np.uint64) * s[l].astype(np.uint64) + M) % np.uint64(q)).astype(np.uint32)
            queries.append(q_)
            evks.append(evk)
            secrets.append(s)
            rgsws.append(np.stack([synth.toy_rgsw(920 + c, st, (j >> st) & 1, s, L, N, primes, ell)
                                   for st in range(D1.bit_length() - 1)]))
        B = len(picks)
        qd, ed, rd = to_dev(np.stack(queries)), to_dev(np.stack(evks)), to_dev(np.stack(rgsws))
        sel = torch.full((B, D0, 2, L, N), -1, dtype=torch.int32, device="cuda")
        rows = torch.full((B, D1, 2, L, N), -1, dtype=torch.int32, device="cuda")
        ref = torch.full((B, 2, L, N), -1, dtype=torch.int32, device="cuda")
        g.gpir_expand_query(h.params, B, J, D0, qd, ed, sel)
        g.gpir_rowsel_batch(h.h, B, sel, rows, g.GPIR_PATH_CUDACORE)
        g.gpir_coltor(h.params, B, D1, rows, rd, ref)
        torch.cuda.synchronize()
        want = to_host(ref)
        for path in (g.GPIR_PATH_CUDACORE, g.GPIR_PATH_IMMA, g.GPIR_PATH_TC):
            out = torch.full((B, 2, L, N), -1, dtype=torch.int32, device="cuda")
            sel.fill_(-1)
            rows.fill_(-1)
            g.gpir_pir_batch(h.h, B, J, qd, ed, rd, sel, rows, out, path)
            torch.cuda.synchronize()
            g.gpir_sync(None, 20000)
            assert np.array_equal(to_host(out), want), "path %d" % path
        assert g.lib.gpir_pir_batch(h.h, B, 5, qd.data_ptr(), ed.data_ptr(), rd.data_ptr(), sel.data_ptr(),
                                    rows.data_ptr(), out.data_ptr(), 0, None) == g.GPIR_EINVAL   # 2^5 < D0
        assert g.lib.gpir_pir_batch(h.h, B, J, qd.data_ptr(), ed.data_ptr(), rd.data_ptr(), sel.data_ptr(),
                                    sel.data_ptr(), out.data_ptr(), 0, None) == g.GPIR_EINVAL   # overlap
    finally:
        h.close()
    for c, (i, j) in enumerate(picks):
        for l, q in enumerate(primes):
            a = want[c, 0, l].astype(np.uint64)
            b = want[c, 1, l].astype(np.uint64)
            m = (b + np.uint64(q) - (a * secrets[c][l].astype(np.uint64)) % np.uint64(q)) % np.uint64(q)
            assert np.array_equal(m, (db[i, j, l].astype(np.uint64) * np.uint64(1 << J)) % np.uint64(q))


def test_pir_batch_replays_from_a_cuda_graph(g):
    """After one warm-up call (tables, workspaces and kernel attributes exist),
    gpir_pir_batch can be captured into a CUDA graph; replays give the result
    of a direct call."""
    import torch
    from tests.gpu_util import DbHandle, to_dev
    N, L, D0, D1, J, B = 512, 2, 32, 8, 5, 3
    primes = P28
    ell = oracle.gadget_digits(primes)
    db = synth.uniform_residues(931, synth.TAG_DB, (D0, D1, L, N), primes, limb_axis=2)
    h = DbHandle(g, db, N, primes, path_mask=g.GPIR_PATH_TC)
    try:
        query = to_dev(synth.uniform_residues(932, eu.TAG_QUERY, (B, 2, L, N), primes, limb_axis=2))
        evk = to_dev(synth.uniform_residues(933, eu.TAG_EVK, (B, J, ell, 2, L, N), primes, limb_axis=4))
        rgsw = to_dev(synth.uniform_residues(934, synth.TAG_RGSW, (B, 3, 2 * ell, 2, L, N), primes, limb_axis=4))
        sel = torch.empty((B, D0, 2, L, N), dtype=torch.int32, device="cuda")
        rows = torch.empty((B, D1, 2, L, N), dtype=torch.int32, device="cuda")
        want = torch.empty((B, 2, L, N), dtype=torch.int32, device="cuda")
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            g.gpir_pir_batch(h.h, B, J, query, evk, rgsw, sel, rows, want, g.GPIR_PATH_TC, s)   # warm-up
        s.synchronize()
        out = torch.full((B, 2, L, N), -1, dtype=torch.int32, device="cuda")
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            g.gpir_pir_batch(h.h, B, J, query, evk, rgsw, sel, rows, out, g.GPIR_PATH_TC,
                             torch.cuda.current_stream())
        for _ in range(2):
            out.fill_(-1)
            graph.replay()
            torch.cuda.synchronize()
            assert torch.equal(out, want)
        g.gpir_sync(None, 20000)
    finally:
        h.close()


def test_expand_degenerate_cases(g):
    """n_out = 1 with J = 3 (every stage computes only index 0, no X^(-2^j)
    output) against the oracle; an all-zero query and keys expand to zeros."""
    primes = P28
    N, L, J = 256, 2, 3
    ell = oracle.gadget_digits(primes)
    query = synth.uniform_residues(941, eu.TAG_QUERY, (2, 2, L, N), primes, limb_axis=2)
    evk = synth.uniform_residues(942, eu.TAG_EVK, (2, J, ell, 2, L, N), primes, limb_axis=4)
    got = _gpu_expand(g, primes, N, query, evk, 1)
    for c in range(2):
        assert np.array_equal(got[c], oracle.expand_query(query[c], evk[c], primes, 1))
    zq = np.zeros_like(query)
    ze = np.zeros_like(evk)
    assert not _gpu_expand(g, primes, N, zq, ze, 8).any()
