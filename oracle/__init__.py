"""CPU oracle for RowSel, the encrypted row-selection step of batched lattice PIR.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously correct
restatement of what RowSel computes, written from the GPIR paper
(arXiv 2604.04696): Sec. 2.2 (RowSel), the GEMM formulation of Sec. 2.3 and
its batched form in Sec. 5.1.1, plus the negacyclic NTT facts of Sec. 2.4.1
that the self-checks rely on.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import it. The GPU product path never imports, links or
calls anything here, and nothing here imports the GPU package.

Every function works in exact integer arithmetic (numpy uint64 / Python int).

Pins (see tests/test_oracle_pins.py): schoolbook negacyclic multiplication vs
NTT on tiny rings and at N=2048, one-hot row selection, a toy noiseless RLWE
selection, linearity in both arguments, closed forms (all q-1, all-ones, zero),
and big-integer brute force on tiny shapes. No function is "parity unpinned".
"""

from .ring import (is_prime, ntt_friendly_primes, primitive_root, psi_2n,
                   ntt_negacyclic, intt_negacyclic, schoolbook_negacyclic)
from .rowsel import rowsel, rowsel_output, rlwe_decrypt_ntt

__all__ = [
    "is_prime", "ntt_friendly_primes", "primitive_root", "psi_2n",
    "ntt_negacyclic", "intt_negacyclic", "schoolbook_negacyclic",
    "rowsel", "rowsel_output", "rlwe_decrypt_ntt",
]
