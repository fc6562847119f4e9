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
