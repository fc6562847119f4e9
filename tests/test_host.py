"""Host-side logic without a GPU: sizes, the input generator, the C ABI's
exported symbols and its argument checks."""

import ctypes
import json
import os
import re

import numpy as np
import pytest

import synth
from paper_2604_04696_gb300 import sizes

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _gold(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


def test_sizes_match_paper():
    g = _gold("paper_sizes.json")
    assert sizes.poly_bytes(4096, 4) == g["a_poly_bytes"]["value"]
    assert sizes.ct_bytes(4096, 4) == g["ct_bytes"]["value"]
    assert sizes.db_bytes(1, 1, 4096, 4) == g["record_poly_bytes"]["value"]
    assert sizes.raw_record_bytes(4096, 32) == g["record_raw_bytes"]["value"]
    assert sizes.query_ct_bytes(32, 256, 4096, 4) == g["expanded_cts_batch32"]["value"]
    assert sizes.naive_transpose_bytes(32, 256, 512, 4096, 4) == g["transpose_traffic_2gb_batch32"]["value"]
    assert sizes.db_bytes(1, 1, 4096, 4) // sizes.raw_record_bytes(4096, 32) == g["storage_overhead"]["value"]
    # 2 GB of raw records at 16 KB each with D0 = 256 gives D1 = 512
    assert (2 << 30) // sizes.raw_record_bytes(4096, 32) // 256 == 512


def test_workload_byte_counts():
    # 4 GiB NTT-form DB at N=4096, 2 limbs, D0=1024, D1=128; 8 GiB of selection cts at B=128
    assert sizes.db_bytes(1024, 128, 4096, 2) == 4 << 30
    assert sizes.query_ct_bytes(128, 1024, 4096, 2) == 8 << 30
    assert sizes.out_bytes(128, 128, 4096, 2) == 1 << 30
    assert sizes.db_bytes(256, 64, 4096, 2) == 512 << 20
    assert sizes.rowsel_modmacs(128, 1024, 128, 4096, 2) == 274877906944


def test_splitmix64_published_vectors():
    g = _gold("splitmix64_vectors.json")
    for key, want in g.items():
        if not key.startswith("seed_"):
            continue
        s = int(key[5:])
        got = []
        for _ in range(len(want)):
            s = (s + synth.GAMMA) & ((1 << 64) - 1)
            got.append(synth.mix64(s))
        assert got == want


def test_counter_stream_is_random_access():
    a = synth.uniform_u64(5, 2, 0, 1000)
    b = synth.uniform_u64(5, 2, 400, 100)
    assert np.array_equal(a[400:500], b)
    key = synth.stream_key(5, 2)
    assert int(a[7]) == synth.mix64(key + 8 * synth.GAMMA)
    assert not np.array_equal(synth.uniform_u64(5, 3, 0, 10), a[:10])


def test_residues_in_range_and_limb_mapping():
    primes = (17, 41)
    x = synth.uniform_residues(3, 1, (3, 2, 8), primes, limb_axis=1)
    assert x[:, 0].max() < 17 and x[:, 1].max() < 41
    v = synth.uniform_u64(3, 1, 0, 48).reshape(3, 2, 8)
    assert np.array_equal(x[:, 0], (v[:, 0] % 17).astype(np.uint32))
    assert np.array_equal(x[:, 1], (v[:, 1] % 41).astype(np.uint32))


def test_residues_roughly_uniform():
    q = synth.PRIMES_28[0]
    x = synth.uniform_residues(0, 2, (1, 200000), (q,), limb_axis=0).astype(np.float64).ravel()
    assert abs(x.mean() / q - 0.5) < 0.005
    hist = np.histogram(x, bins=16, range=(0, q))[0]
    assert hist.min() > 0.9 * 200000 / 16


# ---- C ABI (library loads on a CPU host; no call here touches CUDA) ---------

@pytest.fixture(scope="module")
def g():
    from paper_2604_04696_gb300 import _build
    _build.build()
    from paper_2604_04696_gb300 import gpir
    return gpir


def test_every_header_symbol_is_exported(g):
    with open(os.path.join(ROOT, "include", "gpir.h")) as fh:
        hdr = fh.read()
    declared = set(re.findall(r"\b(gpir_[a-z_0-9]+)\s*\(", hdr))
    assert "gpir_rowsel_batch" in declared and len(declared) >= 15
    for name in sorted(declared):
        assert hasattr(g.lib, name), name


def test_params_checks(g):
    q0, q1 = synth.PRIMES_28
    p = g.gpir_params_create(4096, [q0, q1])
    assert p.value
    g.gpir_params_destroy(p)
    bad = [
        (4096, [q0 + 2]),                 # not prime
        (4096, [268369921 + 8192 * 0 + 4096]),  # not 1 mod 2N
        (3000, [q0]),                     # N not a power of two
        (2, [17]),                        # N below the minimum
        (131072, [q0]),                   # N above the maximum
        (4096, [(1 << 28) + 8193]),       # prime too wide
        (4096, []),                       # no limbs
        (4096, [q0] * 9),                 # too many limbs
    ]
    for n, primes in bad:
        with pytest.raises(g.GpirError) as ei:
            g.gpir_params_create(n, primes)
        assert ei.value.code == g.GPIR_EINVAL
    assert g.gpir_params_create(4, [17, 41]).value
    assert g.gpir_params_create(65536, [786433]).value   # 786433 = 12 * 2^16 + 1, prime


def test_strerror_and_version(g):
    assert g.gpir_version() == 100
    for code in (g.GPIR_OK, g.GPIR_EINVAL, g.GPIR_ERANGE, g.GPIR_ENOMEM, g.GPIR_ECUDA, g.GPIR_ETIMEOUT,
                 g.GPIR_ENOTSUP):
        assert g.gpir_strerror(code) != "unknown gpir error"
    assert g.gpir_strerror(-99) == "unknown gpir error"


def test_null_arguments_rejected(g):
    assert g.lib.gpir_rowsel_batch(None, 1, None, None, 0, None) == g.GPIR_EINVAL
    assert g.lib.gpir_rowsel_multi(None, 0, 0, None) == g.GPIR_EINVAL
    assert g.lib.gpir_db_upload(None, 1, 1, None, 0, 0, None, None) == g.GPIR_EINVAL
    assert g.lib.gpir_db_free(None) == g.GPIR_OK


def test_slot_sampling_matches_full_tensors():
    primes = synth.PRIMES_28
    B, D0, D1, L, N = 3, 5, 4, 2, 16
    ct = synth.ct_tensor(7, B, D0, L, N, primes)
    db = synth.db_tensor(7, D0, D1, L, N, primes)
    slots = [(0, 3), (1, 15), (1, 0)]
    cs = synth.ct_slots(7, B, D0, L, N, primes, slots)
    ds = synth.db_slots(7, D0, D1, L, N, primes, slots)
    for k, (l, t) in enumerate(slots):
        assert np.array_equal(cs[..., k], ct[:, :, :, l, t])
        assert np.array_equal(ds[..., k], db[:, :, l, t])


def test_tree_and_pipeline_argument_errors_on_the_host(g):
    """ColTor, ExpandQuery and the one-call server step check their arguments
    before any CUDA call (no GPU here): fake, non-overlapping addresses."""
    P28 = [268369921, 268361729]
    p = g.gpir_params_create(64, P28)
    try:
        A, B, C = 1 << 40, 2 << 40, 3 << 40
        col, exq = g.lib.gpir_coltor, g.lib.gpir_expand_query
        for d1 in (0, 1, 3, 6):
            assert col(p, 1, d1, A, B, C, None) == g.GPIR_EINVAL
        assert col(p, 0, 4, A, B, C, None) == g.GPIR_EINVAL
        assert col(p, 1, 4, None, B, C, None) == g.GPIR_EINVAL
        assert col(p, 1, 4, A, B, A + 64, None) == g.GPIR_EINVAL            # out inside the input
        assert exq(p, 1, 2, 5, A, B, C, None) == g.GPIR_EINVAL              # n_out > 2^J
        assert exq(p, 1, 2, 0, A, B, C, None) == g.GPIR_EINVAL
        assert exq(p, 0, 2, 4, A, B, C, None) == g.GPIR_EINVAL
        assert exq(p, 1, 7, 4, A, B, C, None) == g.GPIR_EINVAL              # J > log2 N
        assert exq(p, 1, 2, 4, A, None, C, None) == g.GPIR_EINVAL           # no keys
        assert exq(p, 1, 2, 4, A, B, A + 64, None) == g.GPIR_EINVAL         # out overlaps the query
        assert g.lib.gpir_pir_batch(None, 1, 2, A, B, C, A, B, C, 0, None) == g.GPIR_EINVAL
    finally:
        g.gpir_params_destroy(p)
    for n, primes in [(64, P28 + [268271617]), (8, P28[:1]), (8192, [786433])]:
        p3 = g.gpir_params_create(n, primes)
        try:
            assert g.lib.gpir_coltor(p3, 1, 2, 1 << 40, 2 << 40, 3 << 40, None) == g.GPIR_ENOTSUP
            assert g.lib.gpir_expand_query(p3, 1, 1, 2, 1 << 40, 2 << 40, 3 << 40, None) == g.GPIR_ENOTSUP
        finally:
            g.gpir_params_destroy(p3)


def test_debug_switch_and_environment():
    """gpir_set_debug returns the previous setting; GPIR_DEBUG=1 in the
    environment turns the checks on when the library first reads it."""
    import subprocess
    import sys
    code = ("from paper_2604_04696_gb300 import gpir as g; "
            "a = g.gpir_set_debug(True); b = g.gpir_set_debug(False); c = g.gpir_set_debug(False); print(a, b, c)")
    env = dict(os.environ)
    env.pop("GPIR_DEBUG", None)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, check=True)
    assert r.stdout.split() == ["0", "1", "0"]
    env["GPIR_DEBUG"] = "1"
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, check=True)
    assert r.stdout.split() == ["1", "1", "0"]


def test_batch_limit_rejected_before_any_dereference(g):
    """A batch above GPIR_MAX_BATCH (2 * batch rows would not fit 32-bit row
    indices) is an argument error in every RowSel entry point, found before
    the handle is touched (the fake handle address here is never read)."""
    big = g.GPIR_MAX_BATCH + 1
    fake_db, A, B = 1 << 40, 2 << 40, 3 << 40
    assert g.lib.gpir_rowsel_batch(fake_db, big, A, B, 0, None) == g.GPIR_EINVAL
    assert g.lib.gpir_rowsel_batch_host(fake_db, big, A, B, 0, None) == g.GPIR_EINVAL
    assert g.lib.gpir_rowsel_batch_noalloc(fake_db, big, A, B, None) == g.GPIR_EINVAL
    assert g.lib.gpir_autotune(fake_db, big, A, B, 0, None, None) == g.GPIR_EINVAL
    job = g.gpir_job_t(fake_db, big, 0, A, B)
    assert g.lib.gpir_rowsel_multi(ctypes.pointer(job), 1, 0, None) == g.GPIR_EINVAL


def test_fail_alloc_injection_on_the_host():
    """The allocation-failure hook: GPIR_FAIL_ALLOC=n in the environment (or
    gpir_set_fail_alloc) makes the n-th device allocation fail with
    GPIR_ENOMEM, then disarms. Here (no GPU) the database upload's first
    allocation is the one counted: armed at 1 it returns GPIR_ENOMEM; disarmed,
    the same call reaches the CUDA runtime and fails otherwise."""
    import subprocess
    import sys
    code = (
        "import numpy as np, synth\n"
        "from paper_2604_04696_gb300 import gpir as g\n"
        "P = g.gpir_params_create(16, list(synth.PRIMES_28))\n"
        "db = np.zeros(2 * 2 * 2 * 16, dtype=np.uint32)\n"
        "def up():\n"
        "    import ctypes\n"
        "    h = ctypes.c_void_p()\n"
        "    return g.lib.gpir_db_upload(P, 2, 2, db.ctypes.data, 0, 1, None, ctypes.byref(h))\n"
        "first = up()\n"                       # env armed at 1: this one fails
        "second = up()\n"                      # disarmed
        "prev = g.gpir_set_fail_alloc(2)\n"
        "third = up()\n"                       # countdown 2 -> 1: real allocation attempt
        "fourth = up()\n"                      # the 2nd one: injected
        "fifth = up()\n"
        "print(first, second, prev, third, fourth, fifth, g.gpir_set_fail_alloc(0))\n")
    env = dict(os.environ)
    env["GPIR_FAIL_ALLOC"] = "1"
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, check=True)
    first, second, prev, third, fourth, fifth, last = [int(x) for x in r.stdout.split()]
    ENOMEM = -3
    assert first == ENOMEM and prev == 0 and fourth == ENOMEM and last == 0
    assert second != ENOMEM and third != ENOMEM and fifth != ENOMEM
