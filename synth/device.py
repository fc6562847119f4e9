"""Client-side toy query encoding on the device, for driving and checking the
server at full size (no RowSel arithmetic here).

The uniform residues come from the device copy of the synthetic-input
generator, passed in as `fill` (the binding's gpir_fill_uniform), so this
module imports nothing of the library.
"""

import torch

from .gen import TAG_MASK, TAG_SECRET


def toy_rlwe_query(fill, params_ptr, D0, L, N, primes, istar, seed, stream=None):
    """Noiseless toy RLWE one-hot query in the NTT domain, made on the device:
    ct_i = (a_i, a_i (.) s + [i == istar]) mod q_l with a_i, s uniform (the NTT
    of the constant 1 is all ones). Returns (ct [D0][2][L][N] int32 on the
    device, s [L][N] int64 on the device)."""
    a = torch.empty(D0 * L * N, dtype=torch.int32, device="cuda")
    s = torch.empty(L * N, dtype=torch.int32, device="cuda")
    fill(a, a.numel(), 0, seed, TAG_MASK, params_ptr, N, stream)
    fill(s, s.numel(), 0, seed, TAG_SECRET, params_ptr, N, stream)
    a = a.view(D0, L, N).long()
    s = s.view(L, N).long()
    q = torch.tensor(list(primes), dtype=torch.int64, device="cuda").view(1, L, 1)
    b = (a * s.unsqueeze(0)) % q
    b[istar] = (b[istar] + 1) % q[0]
    ct = torch.stack([a, b], dim=1).to(torch.int32).contiguous()
    return ct, s
