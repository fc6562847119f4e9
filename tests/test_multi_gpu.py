"""Multi-job RowSel (several resident databases of uneven shape in one call)
and CUDA-graph plans, bit-exact against the oracle."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from tests import gpu_util
    return gpu_util.lib()


def _problems(n, N=256, L=2, seed=500):
    primes = synth.PRIMES_28[:L]
    rng = np.random.default_rng(seed)
    shapes = [(int(rng.integers(1, 6)), int(rng.integers(1, 300)), int(rng.integers(1, 140))) for _ in range(n)]
    out = []
    for k, (B, D0, D1) in enumerate(shapes):
        ct, db = synth.ct_tensor(seed + k, B, D0, L, N, primes), synth.db_tensor(seed + k, D0, D1, L, N, primes)
        out.append((B, D0, D1, ct, db))
    return out, primes


@pytest.mark.parametrize("path,njobs", [(4, 3), (4, 11), (1, 3), (0, 4)])
def test_multi_matches_oracle(g, path, njobs):
    import torch
    from tests.gpu_util import to_dev, to_host
    if path and g.gpir_num_variants(path) == 0:
        pytest.skip("path not built")
    N = 256
    probs, primes = _problems(njobs, N=N, seed=500 + njobs)
    params = g.gpir_params_create(N, list(primes))
    handles, jobs, outs, wants = [], [], [], []
    try:
        for B, D0, D1, ct, db in probs:
            h = g.gpir_db_upload(params, D0, D1, to_dev(db), True, 0)
            handles.append(h)
            out = torch.full((B, D1, 2, len(primes), N), -1, dtype=torch.int32, device="cuda")
            ctd = to_dev(ct)
            jobs.append((h, B, ctd, out))
            outs.append(out)
            wants.append(oracle.rowsel(ct, db, list(primes)))
        g.gpir_rowsel_multi(jobs, path)
        torch.cuda.synchronize()
        g.gpir_sync(None, 30000)
        for k, (out, want) in enumerate(zip(outs, wants)):
            assert np.array_equal(to_host(out), want), "job %d" % k
    finally:
        for h in handles:
            g.gpir_db_free(h)
        g.gpir_params_destroy(params)


@pytest.mark.parametrize("path", [4, 1])
def test_graph_replay_after_refill(g, path):
    import torch
    from tests.gpu_util import to_dev, to_host
    if g.gpir_num_variants(path) == 0:
        pytest.skip("path not built")
    N = 128
    probs, primes = _problems(3, N=N, seed=900)
    params = g.gpir_params_create(N, list(primes))
    handles, jobs, outs, cts = [], [], [], []
    stream = torch.cuda.Stream()
    graph = None
    try:
        for B, D0, D1, ct, db in probs:
            h = g.gpir_db_upload(params, D0, D1, to_dev(db), True, 0)
            handles.append(h)
            out = torch.full((B, D1, 2, len(primes), N), -1, dtype=torch.int32, device="cuda")
            ctd = to_dev(ct)
            cts.append(ctd)
            jobs.append((h, B, ctd, out))
            outs.append(out)
        with torch.cuda.stream(stream):
            graph = g.gpir_graph_create(jobs, path, stream)
        for rep in range(2):
            wants = []
            for k, (B, D0, D1, _ct, db) in enumerate(probs):
                new_ct = synth.ct_tensor(7000 + 10 * rep + k, B, D0, len(primes), N, primes)
                cts[k].copy_(to_dev(new_ct))
                outs[k].fill_(-1)
                wants.append(oracle.rowsel(new_ct, db, list(primes)))
            torch.cuda.synchronize()
            g.gpir_graph_launch(graph, stream)
            stream.synchronize()
            g.gpir_sync(stream, 30000)
            for k, want in enumerate(wants):
                assert np.array_equal(to_host(outs[k]), want), "replay %d job %d" % (rep, k)
    finally:
        if graph is not None:
            g.gpir_graph_destroy(graph)
        for h in handles:
            g.gpir_db_free(h)
        g.gpir_params_destroy(params)


def test_graph_survives_workspace_growth_on_its_stream(g):
    """A graph owns its workspace: after a larger RowSel on the stream the
    graph was created on (which grows and replaces that stream's workspace),
    replaying the graph is still bit-exact."""
    import torch
    from tests.gpu_util import to_dev, to_host
    if g.gpir_num_variants(4) == 0:
        pytest.skip("path not built")
    N, primes = 128, synth.PRIMES_28
    L = len(primes)
    B, D0, D1 = 2, 70, 33
    ct, db = synth.ct_tensor(951, B, D0, L, N, primes), synth.db_tensor(951, D0, D1, L, N, primes)
    params = g.gpir_params_create(N, list(primes))
    h = g.gpir_db_upload(params, D0, D1, to_dev(db), True, 0)
    stream = torch.cuda.Stream()
    graph = None
    try:
        ctd = to_dev(ct)
        out = torch.full((B, D1, 2, L, N), -1, dtype=torch.int32, device="cuda")
        graph = g.gpir_graph_create([(h, B, ctd, out)], 4, stream)
        big_B = 40
        big_ct = to_dev(synth.ct_tensor(952, big_B, D0, L, N, primes))
        big_out = torch.empty((big_B, D1, 2, L, N), dtype=torch.int32, device="cuda")
        g.gpir_set_variant(h, big_B, 4, 1)                # two-pass form: workspace 2x the ciphertexts
        g.gpir_rowsel_batch(h, big_B, big_ct, big_out, 4, stream)
        stream.synchronize()
        new_ct = synth.ct_tensor(953, B, D0, L, N, primes)
        ctd.copy_(to_dev(new_ct))
        out.fill_(-1)
        torch.cuda.synchronize()
        g.gpir_graph_launch(graph, stream)
        stream.synchronize()
        g.gpir_sync(stream, 30000)
        assert np.array_equal(to_host(out), oracle.rowsel(new_ct, db, list(primes)))
    finally:
        if graph is not None:
            g.gpir_graph_destroy(graph)
        g.gpir_db_free(h)
        g.gpir_params_destroy(params)


def test_multi_argument_errors(g):
    """gpir_rowsel_multi rejects an output that overlaps any ciphertext or
    output buffer of the call, and buffers not 16-byte aligned."""
    import torch
    from tests.gpu_util import to_dev
    N, primes = 64, synth.PRIMES_28
    L = len(primes)
    B, D0, D1 = 2, 8, 8
    db = synth.db_tensor(960, D0, D1, L, N, primes)
    params = g.gpir_params_create(N, list(primes))
    h = g.gpir_db_upload(params, D0, D1, to_dev(db), True, 1)
    try:
        ct = torch.zeros(B * D0 * 2 * L * N + 64, dtype=torch.int32, device="cuda")
        out = torch.zeros(2 * B * D1 * 2 * L * N + 64, dtype=torch.int32, device="cuda")
        half = B * D1 * 2 * L * N
        for jobs in ([(h, B, ct, out), (h, B, ct, out[16:])],        # outputs overlap
                     [(h, B, ct, out), (h, B, out[half:], ct)],       # an output is another job's input
                     [(h, B, ct[1:], out)]):                          # 4-byte misaligned input
            with pytest.raises(g.GpirError) as ei:
                g.gpir_rowsel_multi(jobs, 1)
            assert ei.value.code == g.GPIR_EINVAL
        g.gpir_rowsel_multi([(h, B, ct, out), (h, B, ct, out[half:])], 1)    # disjoint outputs, shared input
        torch.cuda.synchronize()
    finally:
        g.gpir_db_free(h)
        g.gpir_params_destroy(params)


def test_multi_job_tensor_memory_launch_with_ring_wrap(g):
    """Five uneven jobs at N = 512 (batches 17 / 33 / 8 / 25 / 3, D0 700 / 130 /
    64 / 257 / 2600, D1 130 / 40 / 64 / 1 / 9): one persistent tensor-memory
    launch, whose 48 MB ring of 2.6 MB entries (the largest job's 41 k-chunks:
    18 entries) wraps 64 times over the jobs' 1152 entries; the last job
    has six 512-row groups, so its epilogue reduces in the middle of each
    unit. Every output equals the same job
    through gpir_rowsel_batch on the tensor-core path, and the oracle on 16
    spread slots of each job."""
    import torch
    from tests.gpu_util import to_host
    if g.gpir_num_variants(g.GPIR_PATH_TC) == 0:
        pytest.skip("tensor-core path not built")
    N, L = 512, 2
    primes = list(synth.PRIMES_28[:L])
    shapes = [(17, 700, 130), (33, 130, 40), (8, 64, 64), (25, 257, 1), (3, 2600, 9)]
    params = g.gpir_params_create(N, primes)
    handles, jobs, outs, refs, data = [], [], [], [], []
    try:
        for k, (B, D0, D1) in enumerate(shapes):
            db = torch.empty((D0, D1, L, N), dtype=torch.int32, device="cuda")
            g.gpir_fill_uniform(db, db.numel(), 0, 40 + k, synth.TAG_DB, params, N)
            h = g.gpir_db_upload(params, D0, D1, db, True, 0)
            handles.append(h)
            ct = torch.empty((B, D0, 2, L, N), dtype=torch.int32, device="cuda")
            g.gpir_fill_uniform(ct, ct.numel(), 0, 40 + k, synth.TAG_CT, params, N)
            out = torch.full((B, D1, 2, L, N), -1, dtype=torch.int32, device="cuda")
            ref = torch.full((B, D1, 2, L, N), -2, dtype=torch.int32, device="cuda")
            g.gpir_rowsel_batch(h, B, ct, ref, g.GPIR_PATH_TC)
            jobs.append((h, B, ct, out))
            outs.append(out)
            refs.append(ref)
            data.append((db, ct))
        g.gpir_rowsel_multi(jobs, g.GPIR_PATH_TC)
        torch.cuda.synchronize()
        g.gpir_sync(None, 30000)
        for k, (B, D0, D1) in enumerate(shapes):
            got = to_host(outs[k])
            assert np.array_equal(got, to_host(refs[k])), "job %d differs from its single-job call" % k
            db, ct = data[k]
            for s in range(16):
                l, t = s % L, (s * 67 + k * 5) % N
                want = oracle.rowsel(to_host(ct[:, :, :, l:l + 1, t:t + 1].contiguous()),
                                     to_host(db[:, :, l:l + 1, t:t + 1].contiguous()), [primes[l]])
                assert np.array_equal(got[:, :, :, l:l + 1, t:t + 1], want), "job %d slot (%d, %d)" % (k, l, t)
    finally:
        for h in handles:
            g.gpir_db_free(h)
        g.gpir_params_destroy(params)


def test_multi_job_same_database_twice(g):
    """Two jobs on one database (different batches, ciphertexts and outputs)
    and a third on another, in one tensor-memory launch, against the oracle."""
    import torch
    from tests.gpu_util import to_dev, to_host
    if g.gpir_num_variants(g.GPIR_PATH_TC) == 0:
        pytest.skip("tensor-core path not built")
    N, L = 64, 2
    primes = list(synth.PRIMES_28[:L])
    params = g.gpir_params_create(N, primes)
    dbA = synth.db_tensor(610, 150, 80, L, N, primes)
    dbB = synth.db_tensor(611, 70, 20, L, N, primes)
    hA = g.gpir_db_upload(params, 150, 80, to_dev(dbA), True, 0)
    hB = g.gpir_db_upload(params, 70, 20, to_dev(dbB), True, 0)
    try:
        specs = [(hA, dbA, 20, 150, 80, 612), (hA, dbA, 9, 150, 80, 613), (hB, dbB, 12, 70, 20, 614)]
        jobs, outs, wants, keep = [], [], [], []
        for h, db, B, D0, D1, seed in specs:
            ct = synth.ct_tensor(seed, B, D0, L, N, primes)
            ctd = to_dev(ct)
            out = torch.full((B, D1, 2, L, N), -1, dtype=torch.int32, device="cuda")
            jobs.append((h, B, ctd, out))
            keep.append(ctd)
            outs.append(out)
            wants.append(oracle.rowsel(ct, db, primes))
        g.gpir_rowsel_multi(jobs, g.GPIR_PATH_TC)
        torch.cuda.synchronize()
        g.gpir_sync(None, 30000)
        for k, (out, want) in enumerate(zip(outs, wants)):
            assert np.array_equal(to_host(out), want), "job %d" % k
    finally:
        g.gpir_db_free(hA)
        g.gpir_db_free(hB)
        g.gpir_params_destroy(params)
