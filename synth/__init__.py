"""Seeded synthetic inputs for RowSel and ColTor, shared by the oracle tests and the GPU path.

This module holds no RowSel or ColTor arithmetic (the toy RLWE / RGSW
encryptions are client-side inputs). It draws uniform residues from a
counter-based generator so any element can be produced independently and the
same stream can be reproduced on the host and on the device.

Generator: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based stream:
    key      = mix64(seed * GAMMA  XOR  (tag + 1) * TAGMUL)
    value(i) = mix64(key + (i + 1) * GAMMA)
with mix64 the SplitMix64 output function (xor-shift 30/27/31 and the two
published odd multipliers) and GAMMA = 0x9E3779B97F4A7C15.
A residue mod q is value(i) mod q (bias below 2^-36 for q < 2^28).
"""

from .gen import (GAMMA, mix64, stream_key, uniform_u64, uniform_residues, residues_at,
                  uniform_u64_at, ct_slots, db_slots,
                  ct_tensor, db_tensor, TAG_DB, TAG_CT, TAG_SECRET, TAG_MASK,
                  toy_rlwe_selection, config_shapes, CONFIGS, PRIMES_28,
                  TAG_RGSW, TAG_COLTOR, TAG_RECORD, TAG_EVK, TAG_QUERY, TAG_MESSAGE,
                  toy_rgsw, toy_coltor_inputs)

__all__ = ["GAMMA", "mix64", "stream_key", "uniform_u64", "uniform_residues", "residues_at",
           "uniform_u64_at", "ct_slots", "db_slots",
           "ct_tensor", "db_tensor", "TAG_DB", "TAG_CT", "TAG_SECRET", "TAG_MASK",
           "toy_rlwe_selection", "config_shapes", "CONFIGS", "PRIMES_28",
           "TAG_RGSW", "TAG_COLTOR", "TAG_RECORD", "TAG_EVK", "TAG_QUERY", "TAG_MESSAGE",
           "toy_rgsw", "toy_coltor_inputs"]
