"""Run ExpandQuery on one seeded synthetic problem: a fixed launch sequence for
profilers (ncu -k expand_stage_kernel -s <skip> -c <count>) and a quick timing
with CUDA events.

    python paper_2604_04696_gb300/tools/expand_case.py --batch 32 --stages 9 --n-out 274 --n 4096 --limbs 2 --reps 3

Launch sequence: two fill kernels (queries, evaluation keys), then `reps`
warm-up calls and `reps` timed ones; each call launches one stage kernel per
tree level (`stages` launches). Inputs are uniform residues drawn on the
device with gpir_fill_uniform (seed 9).
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
    ap.add_argument("--stages", type=int, default=9)
    ap.add_argument("--n-out", type=int, default=274)
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--limbs", type=int, default=2)
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)

    import torch
    import synth
    from paper_2604_04696_gb300 import gpir as g

    params = g.gpir_params_create(a.n, list(synth.PRIMES_28[:a.limbs]))
    ell = g.gpir_coltor_gadget_digits(params)
    query = torch.empty(a.batch * 2 * a.limbs * a.n, dtype=torch.int32, device="cuda")
    evk = torch.empty(a.batch * a.stages * ell * 2 * a.limbs * a.n, dtype=torch.int32, device="cuda")
    out = torch.empty(a.batch * a.n_out * 2 * a.limbs * a.n, dtype=torch.int32, device="cuda")
    g.gpir_fill_uniform(query, query.numel(), 0, 9, synth.TAG_QUERY, params, a.n)
    g.gpir_fill_uniform(evk, evk.numel(), 0, 9, synth.TAG_EVK, params, a.n)
    for _ in range(a.reps):
        g.gpir_expand_query(params, a.batch, a.stages, a.n_out, query, evk, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        g.gpir_expand_query(params, a.batch, a.stages, a.n_out, query, evk, out)
    e1.record()
    torch.cuda.synchronize()
    g.gpir_sync(None, 60000)
    print("expand B=%d J=%d n_out=%d N=%d L=%d ell=%d: %.4f ms per call (%d stage launches)"
          % (a.batch, a.stages, a.n_out, a.n, a.limbs, ell, e0.elapsed_time(e1) / a.reps, a.stages))
    g.gpir_params_destroy(params)


if __name__ == "__main__":
    main()
