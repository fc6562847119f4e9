"""Plant plausible mistakes in copies of the oracle (on the CPU) and check
that at least one pin rejects each, so the pins can tell right from wrong."""

import numpy as np
import pytest

import oracle
from tests import pins


def _base(ct, db, primes, variant):
    ct = np.asarray(ct)
    db = np.asarray(db)
    B, D0, _, L, T = ct.shape
    D1 = db.shape[1]
    out = np.empty((B, D1, 2, L, T), dtype=np.uint32)
    for l in range(L):
        q = np.uint64(primes[0] if variant == "limb0_prime" else primes[l])
        acc = np.zeros((B, D1, 2, T), dtype=np.uint64)
        for i in range(D0):
            rsel = 1 - np.arange(2) if variant == "swap_poly" else np.arange(2)
            sel = ct[:, i, :, l, :][:, rsel].astype(np.uint64)
            ii = (i + 1) % D0 if variant == "row_shift" else i
            row = db[ii, :, l, :].astype(np.uint64)
            if variant == "slot_shift":
                row = np.roll(row, 1, axis=-1)
            prod = sel[:, None, :, :] * row[None, :, None, :]
            if variant == "u32_wrap":
                acc = (acc + prod) & np.uint64(0xFFFFFFFF)
            else:
                acc += prod % q
        res = acc if variant in ("no_final_mod",) else acc % q
        out[:, :, :, l, :] = res.astype(np.uint32)
    return out


MUTANTS = ["limb0_prime", "swap_poly", "row_shift", "slot_shift", "u32_wrap", "no_final_mod"]


def test_unmutated_copy_passes_all_pins():
    f = lambda ct, db, primes: _base(ct, db, primes, "none")
    for pin in pins.ALL_PINS:
        pin(f)


@pytest.mark.parametrize("variant", MUTANTS)
def test_mutant_is_caught(variant):
    f = lambda ct, db, primes: _base(ct, db, primes, variant)
    caught = []
    for pin in pins.ALL_PINS:
        try:
            pin(f)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, "no pin caught mutant %s" % variant
