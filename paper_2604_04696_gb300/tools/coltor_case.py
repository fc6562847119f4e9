"""Run ColTor on one seeded synthetic problem: a fixed launch sequence for
profilers (ncu -k coltor_stage_kernel -s <skip> -c <count>) and a quick timing
with CUDA events.

    python paper_2604_04696_gb300/tools/coltor_case.py --batch 32 --d1 64 --n 4096 --limbs 2 --reps 3

Launch sequence: two fill kernels (ciphertexts, RGSW rows), then `reps`
warm-up ColTor calls and `reps` timed ones; each call launches one stage
kernel per tournament level (log2 d1 launches). Inputs are uniform residues
drawn on the device with gpir_fill_uniform (seed 9).
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
    ap.add_argument("--d1", type=int, default=64)
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--limbs", type=int, default=2)
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)

    import torch
    import synth
    from paper_2604_04696_gb300 import gpir as g

    params = g.gpir_params_create(a.n, list(synth.PRIMES_28[:a.limbs]))
    ell = g.gpir_coltor_gadget_digits(params)
    stages = a.d1.bit_length() - 1
    ct = torch.empty(a.batch * a.d1 * 2 * a.limbs * a.n, dtype=torch.int32, device="cuda")
    rgsw = torch.empty(a.batch * stages * 2 * ell * 2 * a.limbs * a.n, dtype=torch.int32, device="cuda")
    out = torch.empty(a.batch * 2 * a.limbs * a.n, dtype=torch.int32, device="cuda")
    g.gpir_fill_uniform(ct, ct.numel(), 0, 9, synth.TAG_COLTOR, params, a.n)
    g.gpir_fill_uniform(rgsw, rgsw.numel(), 0, 9, synth.TAG_RGSW, params, a.n)
    for _ in range(a.reps):
        g.gpir_coltor(params, a.batch, a.d1, ct, rgsw, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        g.gpir_coltor(params, a.batch, a.d1, ct, rgsw, out)
    e1.record()
    torch.cuda.synchronize()
    g.gpir_sync(None, 60000)
    print("coltor B=%d D1=%d N=%d L=%d ell=%d: %.4f ms per call (%d stage launches)"
          % (a.batch, a.d1, a.n, a.limbs, ell, e0.elapsed_time(e1) / a.reps, stages))
    g.gpir_params_destroy(params)


if __name__ == "__main__":
    main()
