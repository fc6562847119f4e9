"""Run RowSel on one seeded synthetic problem of any shape: a fixed launch
sequence for profilers (ncu -k <kernel> -s <skip> -c <count>) and a quick
timing with CUDA events.

    python paper_2604_04696_gb300/tools/rowsel_case.py --batch 32 --d0 256 --d1 64 --n 4096 --limbs 2 \\
        --path tc --variant 0 --reps 3

Launch sequence: two fill kernels (DB, ciphertexts), the upload's range check
and packing kernels, then `reps` warm-up RowSel launches and `reps` timed ones.
Inputs are drawn on the device with gpir_fill_uniform (tags 1 and 2, seed 1).
"""

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PATHS = {"cc": 1, "imma": 2, "tc": 4}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--d0", type=int, default=256)
    ap.add_argument("--d1", type=int, default=64)
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--limbs", type=int, default=2)
    ap.add_argument("--path", choices=sorted(PATHS), default="tc")
    ap.add_argument("--variant", type=int, default=-1, help="tile variant (-1: the library default)")
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)

    import torch
    import synth
    from paper_2604_04696_gb300 import gpir as g

    path = PATHS[a.path]
    params = g.gpir_params_create(a.n, list(synth.PRIMES_28[:a.limbs]))
    db = torch.empty(a.d0 * a.d1 * a.limbs * a.n, dtype=torch.int32, device="cuda")
    g.gpir_fill_uniform(db, db.numel(), 0, 1, synth.TAG_DB, params, a.n)
    h = g.gpir_db_upload(params, a.d0, a.d1, db, True, path)
    del db
    torch.cuda.empty_cache()
    ct = torch.empty(a.batch * a.d0 * 2 * a.limbs * a.n, dtype=torch.int32, device="cuda")
    g.gpir_fill_uniform(ct, ct.numel(), 0, 1, synth.TAG_CT, params, a.n)
    out = torch.empty(a.batch * a.d1 * 2 * a.limbs * a.n, dtype=torch.int32, device="cuda")
    if a.variant >= 0:
        g.gpir_set_variant(h, a.batch, path, a.variant)
    for _ in range(a.reps):
        g.gpir_rowsel_batch(h, a.batch, ct, out, path)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        g.gpir_rowsel_batch(h, a.batch, ct, out, path)
    e1.record()
    torch.cuda.synchronize()
    g.gpir_sync(None, 60000)
    print("rowsel %s variant %d: %.4f ms per launch" % (a.path, g.gpir_selected_variant(h, a.batch, path),
                                                           e0.elapsed_time(e1) / a.reps))
    g.gpir_db_free(h)
    g.gpir_params_destroy(params)


if __name__ == "__main__":
    main()
