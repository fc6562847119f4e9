"""The tensor-memory kernel divides its unit, entry and ingest-task indices by
launch constants with one multiply-high, one add and one shift (Granlund and
Montgomery, 1994): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1 and
n / d = (umulhi(n, m) + n) >> l (rowsel_tmem.cu, TmDiv). This restates the
host's choice of (m, l) and the device formula in integers and checks them
against exact division: every divisor the kernel can see, edge dividends and
random ones; a multiplier one too small is caught."""

import random

import pytest


def tm_div(d):
    d = max(d, 1)
    l = 0
    while (1 << l) < d:
        l += 1
    m = ((1 << 32) * ((1 << l) - d)) // d + 1
    return d, m, l


def fast_div(n, dml, m_off=0):
    d, m, l = dml
    t = (n * (m + m_off)) >> 32        # umulhi
    return (t + n) >> l


def dividends(rng, d):
    base = [0, 1, d - 1, d, d + 1, 2 * d - 1, 2 * d, (1 << 31) - 1, 1 << 31, (1 << 32) - 1,
            ((1 << 32) - 1) // d * d, ((1 << 32) - 1) // d * d - 1]
    return [n for n in base if 0 <= n < (1 << 32)] + [rng.randrange(1 << 32) for _ in range(200)]


@pytest.mark.parametrize("block", range(8))
def test_small_divisors_exact(block):
    """Divisors 1..4096 (k-chunk, m-block, n-block, unit-per-entry and slot-group
    counts of realistic shapes)."""
    rng = random.Random(block)
    for d in range(1 + 512 * block, 513 + 512 * block):
        dml = tm_div(d)
        assert 0 < dml[1] < (1 << 32)
        for n in dividends(rng, d):
            assert fast_div(n, dml) == n // d, (d, n)


def test_large_and_power_of_two_divisors_exact():
    rng = random.Random(7)
    ds = [1 << k for k in range(32)] + [(1 << k) + 1 for k in range(1, 32)] + [(1 << k) - 1 for k in range(2, 33)]
    ds += [rng.randrange(1, 1 << 32) for _ in range(300)]
    for d in ds:
        dml = tm_div(d)
        assert 0 < dml[1] <= (1 << 32) - 1
        for n in dividends(rng, d):
            assert fast_div(n, dml) == n // d, (d, n)


def test_multiplier_one_too_small_is_caught():
    """Sensitivity: rounding the multiplier down (m - 1) breaks exactness for
    some divisor and dividend below 2^32."""
    rng = random.Random(3)
    bad = 0
    for d in [3, 5, 7, 11, 13, 96, 640, 1000003]:
        dml = tm_div(d)
        for n in dividends(rng, d):
            if fast_div(n, dml, m_off=-1) != n // d:
                bad += 1
    assert bad > 0
