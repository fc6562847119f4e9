"""Continuous-batching server: every answer is the same alone and in the mix
(bit-exact, tolerance 0), decrypts to the selected DB row, and admission
respects the memory budget."""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from tests import gpu_util
    return gpu_util.lib()


def _setup(g, shapes, N, primes, seed):
    import torch
    from paper_2604_04696_gb300.server import ResidentDb
    from synth.device import toy_rlwe_query
    params = g.gpir_params_create(N, list(primes))
    L = len(primes)
    dbs, db_dev, pools = [], [], []
    for k, (D0, D1) in enumerate(shapes):
        db = torch.empty(D0 * D1 * L * N, dtype=torch.int32, device="cuda")
        g.gpir_fill_uniform(db, db.numel(), 0, seed + k, synth.TAG_DB, params, N)
        h = g.gpir_db_upload(params, D0, D1, db, True, 0)
        dbs.append(ResidentDb(h, D0, D1, N, L))
        db_dev.append(db.view(D0, D1, L, N))
        pool = []
        for qi, istar in enumerate(sorted({0, D0 - 1, D0 // 2})):
            ct, sec = toy_rlwe_query(g.gpir_fill_uniform, params, D0, L, N, primes, istar,
                                     seed * 100 + k * 10 + qi)
            pool.append((istar, ct, ct.cpu().pin_memory(), sec))
        pools.append(pool)
    torch.cuda.synchronize()
    return params, dbs, db_dev, pools


def test_served_answers_equal_alone_and_decrypt(g):
    import torch
    from paper_2604_04696_gb300.server import Request, Server, poisson_arrivals
    N, primes = 256, synth.PRIMES_28
    shapes = [(40, 24), (70, 64), (33, 130)]
    params, dbs, db_dev, pools = _setup(g, shapes, N, primes, 40)
    try:
        rng = np.random.default_rng(3)
        arr = poisson_arrivals(20000.0, 60, seed=4)
        reqs = []
        for i, t in enumerate(arr):
            d = int(rng.integers(0, len(dbs)))
            qi = int(rng.integers(0, len(pools[d])))
            r = Request(i, d, pools[d][qi][2], float(t))
            r.out = None
            reqs.append((r, qi))
        budget = 10 * max(db.req_bytes for db in dbs)
        srv = Server(dbs, budget, max_batch=8, n_streams=2, keep_outputs=True)
        stats = srv.run([r for r, _ in reqs], timeout_s=60)
        assert stats["completed"] == 60 and stats["rejected"] == 0
        assert stats["batches"] < 60 and stats["mean_batch"] > 1.0
        assert stats["max_admitted_bytes"] <= budget
        for r, qi in reqs:
            istar, ct_dev, _, sec = pools[r.db][qi]
            served = r.out.cuda()
            assert decrypt_check(served, sec, db_dev[r.db][istar], primes), r.rid
            alone = torch.full_like(served, -1).unsqueeze(0)
            g.gpir_rowsel_batch(dbs[r.db].h, 1, ct_dev, alone)
            torch.cuda.synchronize()
            assert torch.equal(alone[0], served), r.rid
    finally:
        for d in dbs:
            g.gpir_db_free(d.h)
        g.gpir_params_destroy(params)


def test_admission_budget_and_rejection(g):
    from paper_2604_04696_gb300.server import Request, Server, poisson_arrivals
    N, primes = 128, synth.PRIMES_28
    shapes = [(64, 32), (900, 16)]
    params, dbs, db_dev, pools = _setup(g, shapes, N, primes, 77)
    try:
        budget = 3 * dbs[0].req_bytes            # the second DB's requests never fit
        assert dbs[1].req_bytes > budget
        arr = poisson_arrivals(50000.0, 24, seed=9)
        reqs = [Request(i, i % 2, pools[i % 2][0][2], float(t)) for i, t in enumerate(arr)]
        srv = Server(dbs, budget, max_batch=4, n_streams=2)
        stats = srv.run(reqs, timeout_s=60)
        assert stats["rejected"] == 12 and stats["completed"] == 12
        assert stats["max_admitted_bytes"] <= budget
        assert stats["p99_ms"] >= stats["p50_ms"] > 0
    finally:
        for d in dbs:
            g.gpir_db_free(d.h)
        g.gpir_params_destroy(params)


def decrypt_check(out, s, db_row, primes):
    """out: [D1][2][L][N] int32 (device), s: [L][N] int64, db_row: [D1][L][N] int32.
    True iff b - a (.) s == DB[i*][j] for every j (noiseless toy RLWE)."""
    import torch
    L = s.shape[0]
    q = torch.tensor(list(primes), dtype=torch.int64, device=out.device).view(1, L, 1)
    a = out[:, 0].long()
    b = out[:, 1].long()
    m = (b - (a * s.unsqueeze(0)) % q) % q
    return bool(torch.equal(m, db_row.long()))
