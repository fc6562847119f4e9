"""Run one PIR server step (gpir_pir_batch: ExpandQuery -> RowSel -> ColTor) on
a seeded synthetic problem: a fixed launch sequence for profilers and a quick
timing with CUDA events.

    python paper_2604_04696_gb300/tools/pir_case.py --batch 32 --d0 256 --d1 64 --n 4096 --limbs 2 --reps 3

Launch sequence: fill kernels (DB, queries, keys, RGSW rows), the DB upload's
range check and packing kernels, then `reps` warm-up steps and `reps` timed
ones. Each step: J = ceil(log2 D0) ExpandQuery stage launches, one RowSel
launch (tensor-core path), log2 D1 ColTor stage launches.
"""

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--d0", type=int, default=256)
    ap.add_argument("--d1", type=int, default=64)
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--limbs", type=int, default=2)
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)

    import torch
    import synth
    from paper_2604_04696_gb300 import gpir as g

    B, D0, D1, N, L = a.batch, a.d0, a.d1, a.n, a.limbs
    params = g.gpir_params_create(N, list(synth.PRIMES_28[:L]))
    ell = g.gpir_coltor_gadget_digits(params)
    J = (D0 - 1).bit_length()
    stages = D1.bit_length() - 1
    ctw = 2 * L * N
    db = torch.empty(D0 * D1 * L * N, dtype=torch.int32, device="cuda")
    g.gpir_fill_uniform(db, db.numel(), 0, 1, synth.TAG_DB, params, N)
    h = g.gpir_db_upload(params, D0, D1, db, True, g.GPIR_PATH_TC)
    del db
    query = torch.empty(B * ctw, dtype=torch.int32, device="cuda")
    evk = torch.empty(B * J * ell * ctw, dtype=torch.int32, device="cuda")
    rgsw = torch.empty(B * stages * 2 * ell * ctw, dtype=torch.int32, device="cuda")
    g.gpir_fill_uniform(query, query.numel(), 0, 9, synth.TAG_QUERY, params, N)
    g.gpir_fill_uniform(evk, evk.numel(), 0, 9, synth.TAG_EVK, params, N)
    g.gpir_fill_uniform(rgsw, rgsw.numel(), 0, 9, synth.TAG_RGSW, params, N)
    sel = torch.empty(B * D0 * ctw, dtype=torch.int32, device="cuda")
    rows = torch.empty(B * D1 * ctw, dtype=torch.int32, device="cuda")
    out = torch.empty(B * ctw, dtype=torch.int32, device="cuda")
    step = lambda: g.gpir_pir_batch(h, B, J, query, evk, rgsw, sel, rows, out, g.GPIR_PATH_TC)
    for _ in range(a.reps):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        step()
    e1.record()
    torch.cuda.synchronize()
    g.gpir_sync(None, 60000)
    print("pir step B=%d D0=%d D1=%d N=%d L=%d (J=%d, %d ColTor stages): %.4f ms per step"
          % (B, D0, D1, N, L, J, stages, e0.elapsed_time(e1) / a.reps))
    g.gpir_db_free(h)
    g.gpir_params_destroy(params)


if __name__ == "__main__":
    main()
