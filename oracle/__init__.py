"""CPU oracle for ExpandQuery, RowSel and ColTor, the three server steps of
batched lattice PIR.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously correct
restatement of what ExpandQuery, RowSel and ColTor compute, written from the
GPIR paper (arXiv 2604.04696): Sec. 2.2 (the three phases), the GEMM
formulation of Sec. 2.3
and its batched form in Sec. 5.1.1, the negacyclic NTT facts of Sec. 2.4.1, and
the external-product steps of Sec. 2.5.1 (inverse NTT, Dcp with RNS
reconstruction, forward NTT, multiply-accumulate), shared by the external
product of ColTor and the key switching inside ExpandQuery's Subs.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import it. The GPU product path never imports, links or
calls anything here, and nothing here imports the GPU package.

Every function works in exact integer arithmetic (numpy uint64 / Python int).

Pins (see tests/test_oracle_pins.py, tests/test_coltor_pins.py): schoolbook
negacyclic multiplication vs NTT on tiny rings and at N=2048, one-hot row
selection, a toy noiseless RLWE selection, linearity in both arguments, closed
forms (all q-1, all-ones, zero), big-integer brute force on tiny shapes; for
ColTor: CRT and digit reconstruction identities, the external product's
decryption identity under noiseless toy RGSW encryptions (checked against a
coefficient-domain schoolbook product), and the whole tournament decrypting to
the selected record; for ExpandQuery (tests/test_expand_pins.py): the
automorphism against direct polynomial evaluation and against the NTT-domain
slot permutation, monomial products against schoolbook, Subs decrypting to the
substituted phase under noiseless toy keys, and the whole tree splitting a
message polynomial into its coefficients. No function is "parity unpinned".
"""

from .ring import (is_prime, ntt_friendly_primes, primitive_root, psi_2n,
                   ntt_negacyclic, intt_negacyclic, schoolbook_negacyclic)
from .rowsel import rowsel, rowsel_output, rlwe_decrypt_ntt
from .coltor import (GADGET_LOG_BASE, gadget_digits, crt_centered, balanced_digits, decompose,
                     external_product, cmux, coltor)
from .expand import automorphism_coeffs, automorphism_ntt, monomial_ntt, subs, expand_node, expand_query

__all__ = [
    "is_prime", "ntt_friendly_primes", "primitive_root", "psi_2n",
    "ntt_negacyclic", "intt_negacyclic", "schoolbook_negacyclic",
    "rowsel", "rowsel_output", "rlwe_decrypt_ntt",
    "GADGET_LOG_BASE", "gadget_digits", "crt_centered", "balanced_digits", "decompose",
    "external_product", "cmux", "coltor",
    "automorphism_coeffs", "automorphism_ntt", "monomial_ntt", "subs", "expand_node", "expand_query",
]
