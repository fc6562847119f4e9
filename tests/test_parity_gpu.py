"""GPU RowSel vs the CPU oracle, bit-exact (modular integer work: tolerance 0).

All calls go through the C ABI (libgpir.so) via the ctypes binding."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

PATHS = {"cudacore": 1, "imma": 2, "tc": 4}
PATH_LIST = ["cudacore", "imma", "tc"]


@pytest.fixture(scope="module")
def g():
    from tests import gpu_util
    return gpu_util.lib()


def _avail_paths(g):
    return [name for name, p in PATHS.items() if g.gpir_num_variants(p) > 0]


def _skip_unbuilt(g, path):
    if g.gpir_num_variants(path) == 0:
        pytest.skip("path not built")


def _check_full(g, B, D0, D1, L, N, primes, seed, path, variants=None):
    from tests.gpu_util import DbHandle, to_dev, to_host, make_problem
    _skip_unbuilt(g, path)
    ct, db = make_problem(seed, B, D0, D1, L, N, primes)
    want = oracle.rowsel(ct, db, list(primes))
    h = DbHandle(g, db, N, primes, path_mask=path)
    try:
        ct_d = to_dev(ct)
        vs = variants if variants is not None else [None]
        for v in vs:
            if v is not None:
                g.gpir_set_variant(h.h, B, path, v)
            got = to_host(h.rowsel(ct_d, B, path))
            assert np.array_equal(got, want), "mismatch path %d variant %s: %d of %d differ" % (
                path, v, int((got != want).sum()), want.size)
    finally:
        h.close()


SHAPES = [
    # (B, D0, D1, L, N, primes)                      what it covers
    (1, 16, 16, 1, 2048, synth.PRIMES_28[:1]),      # plain RowSel workload, seed 0
    (3, 40, 24, 2, 64, synth.PRIMES_28),            # ragged rows / cols / clients
    (9, 300, 70, 2, 128, synth.PRIMES_28),          # D0 crosses the 256-row reduction period
    (2, 5, 3, 2, 8, (17, 97)),                      # ring smaller than a warp of slots
    (1, 1, 1, 1, 4, (17,)),                         # degenerate 1 x 1
    (5, 33, 65, 3, 32, (193, 257, 449)),            # three limbs
    (17, 64, 17, 1, 96 * 0 + 64, (268369921,)),     # odd client count
    (18, 130, 70, 2, 512, synth.PRIMES_28),         # ragged m/n blocks; TC digit and output rings wrap
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "B%d_D0%d_D1%d_L%d_N%d" % s[:5])
@pytest.mark.parametrize("path", PATH_LIST)
def test_rowsel_vs_oracle(g, shape, path):
    B, D0, D1, L, N, primes = shape
    seed = 0 if (B, D0, D1, N) == (1, 16, 16, 2048) else 1000 + B + D0
    if g.gpir_num_variants(PATHS[path]) == 0:
        pytest.skip("path not built")
    _check_full(g, B, D0, D1, L, N, primes, seed, PATHS[path])


@pytest.mark.parametrize("B", [6, 17])
@pytest.mark.parametrize("path", PATH_LIST)
def test_every_variant(g, path, B):
    """Every compiled tile variant of every path; B = 17 gives the tensor-core
    kernels two 32-row m-blocks (the SM-pair variant runs as pairs)."""
    p = PATHS[path]
    nv = g.gpir_num_variants(p)
    _check_full(g, B, 70, 40, 2, 64, synth.PRIMES_28, 77 + B, p, variants=list(range(nv)))


TMEM_VARIANTS = [8, 9, 10, 11]    # tensor-memory kernel (12 digit products): single CTA, SM pair, with L2 hints


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "B%d_D0%d_D1%d_L%d_N%d" % s[:5])
def test_tmem_kernel_vs_oracle(g, shape):
    """The tensor-memory kernel (A operand in tensor memory, centred digits,
    12 products per modular MAC) on every parity shape, both forms."""
    B, D0, D1, L, N, primes = shape
    _check_full(g, B, D0, D1, L, N, primes, 2000 + B + D0, PATHS["tc"], variants=TMEM_VARIANTS)


def test_tmem_kernel_many_clients(g):
    """257 clients: 17 m-blocks of 32 rows, the last with 2 rows (the SM-pair
    variants, which need an even count, run the single-CTA form), ragged D0
    and D1, against the oracle."""
    _check_full(g, 257, 100, 70, 2, 32, synth.PRIMES_28, 4257, PATHS["tc"], variants=TMEM_VARIANTS)


@pytest.mark.parametrize("B", [16, 33])
@pytest.mark.parametrize("xy", [("q-1056832", "q-524800"), ("133160903", "q-524800"), ("h", "h+1"),
                                ("q-1", "q-1")])
def test_tmem_extreme_digits_reach_the_bound(g, B, xy):
    """Residues whose centred digits sit at the ends of their ranges, over
    D0 = 2048 rows (four 512-row groups): ciphertext q - 1056832 (digits -64,
    -64, -64, 0) against database q - 524800 (digits -512, -512, 0) drives the
    group sums of 6 of the 12 digit pairs to exactly 2^24; 133160903 puts the
    top ciphertext digit at +64. Result D0 * x * y mod q everywhere. B = 16
    gives one 32-row m-block (single-CTA form even for the pair variant), B =
    33 three (pairs plus a single)."""
    from tests.gpu_util import DbHandle, to_dev, to_host
    _skip_unbuilt(g, PATHS["tc"])
    primes = synth.PRIMES_28
    D0, D1, L, N = 2048, 72, 2, 32
    val = {"q-1056832": lambda q: q - 1056832, "q-524800": lambda q: q - 524800, "133160903": lambda q: 133160903,
           "h": lambda q: (q - 1) // 2, "h+1": lambda q: (q + 1) // 2, "q-1": lambda q: q - 1}
    fx, fy = val[xy[0]], val[xy[1]]
    ct = np.empty((B, D0, 2, L, N), dtype=np.uint32)
    db = np.empty((D0, D1, L, N), dtype=np.uint32)
    for l, q in enumerate(primes):
        ct[:, :, :, l] = fx(q)
        db[:, :, l] = fy(q)
    h = DbHandle(g, db, N, primes, path_mask=PATHS["tc"])
    try:
        ct_d = to_dev(ct)
        for v in TMEM_VARIANTS:
            g.gpir_set_variant(h.h, B, PATHS["tc"], v)
            got = to_host(h.rowsel(ct_d, B, PATHS["tc"]))
            for l, q in enumerate(primes):
                assert np.all(got[:, :, :, l] == (D0 * fx(q) * fy(q)) % q), (v, l)
    finally:
        h.close()


@pytest.mark.parametrize("B,D0", [(5, 2600), (34, 3100)])
def test_tmem_deferred_reduction_across_flushes(g, B, D0):
    """The tensor-memory epilogue sums four 512-row groups before one
    reduction: D0 = 2600 (6 groups, the last partial) and 3100 (7 groups)
    reduce once in the middle of each unit and once at its end. Random
    residues, every tensor-memory variant, against the oracle; B = 34 gives
    three 32-row m-blocks (the pair variants run pairs plus a single)."""
    _check_full(g, B, D0, 70, 2, 16, synth.PRIMES_28, 3000 + D0, PATHS["tc"], variants=TMEM_VARIANTS)


def test_tmem_extreme_digits_over_eight_groups(g):
    """Bound-driving residues (ciphertext q - 1056832, database q - 524800: six
    of the twelve group sums at exactly 2^24) over D0 = 4096 rows, eight
    groups, two deferred reductions per unit: result D0 * x * y mod q."""
    from tests.gpu_util import DbHandle, to_dev, to_host
    _skip_unbuilt(g, PATHS["tc"])
    primes = synth.PRIMES_28
    B, D0, D1, L, N = 16, 4096, 70, 2, 16
    ct = np.empty((B, D0, 2, L, N), dtype=np.uint32)
    db = np.empty((D0, D1, L, N), dtype=np.uint32)
    for l, q in enumerate(primes):
        ct[:, :, :, l] = q - 1056832
        db[:, :, l] = q - 524800
    h = DbHandle(g, db, N, primes, path_mask=PATHS["tc"])
    try:
        ct_d = to_dev(ct)
        for v in TMEM_VARIANTS:
            g.gpir_set_variant(h.h, B, PATHS["tc"], v)
            got = to_host(h.rowsel(ct_d, B, PATHS["tc"]))
            for l, q in enumerate(primes):
                want = (D0 * (q - 1056832) * (q - 524800)) % q
                assert np.all(got[:, :, :, l] == want), (v, l)
    finally:
        h.close()


@pytest.mark.parametrize("path", PATH_LIST)
def test_worst_case_accumulation(g, path):
    """All residues q-1 with D0 = 2048: every product is maximal; result D0 mod q."""
    from tests.gpu_util import DbHandle, to_dev, to_host
    _skip_unbuilt(g, PATHS[path])
    primes = synth.PRIMES_28
    B, D0, D1, L, N = 2, 2048, 8, 2, 32
    ct = np.empty((B, D0, 2, L, N), dtype=np.uint32)
    db = np.empty((D0, D1, L, N), dtype=np.uint32)
    for l, q in enumerate(primes):
        ct[:, :, :, l] = q - 1
        db[:, :, l] = q - 1
    h = DbHandle(g, db, N, primes, path_mask=PATHS[path])
    try:
        got = to_host(h.rowsel(to_dev(ct), B, PATHS[path]))
    finally:
        h.close()
    for l, q in enumerate(primes):
        assert np.all(got[:, :, :, l] == D0 % q)


@pytest.mark.parametrize("path", PATH_LIST)
@pytest.mark.parametrize("a,b", [(0x7F7F80, 0x7F7F80), (0x7F7F80, 0x7F7F7F), (0x7F7F7F, 0x7F7F7F)])
def test_extreme_digit_accumulation(g, path, a, b):
    """Residues whose signed base-256 digits are all at the ends of their range
    (0x7F7F80 -> -128, -128, -128, 1; 0x7F7F7F -> 127, 127, 127, 0), over
    D0 = 2048 rows: every exact partial sum of the digit products reaches its
    bound. The result is D0 * a * b mod q."""
    from tests.gpu_util import DbHandle, to_dev, to_host
    _skip_unbuilt(g, PATHS[path])
    primes = synth.PRIMES_28
    B, D0, D1, L, N = 2, 2048, 8, 2, 32
    ct = np.full((B, D0, 2, L, N), a, dtype=np.uint32)
    db = np.full((D0, D1, L, N), b, dtype=np.uint32)
    h = DbHandle(g, db, N, primes, path_mask=PATHS[path])
    try:
        got = to_host(h.rowsel(to_dev(ct), B, PATHS[path]))
    finally:
        h.close()
    for l, q in enumerate(primes):
        assert np.all(got[:, :, :, l] == (D0 * a * b) % q)


@pytest.mark.parametrize("path", PATH_LIST)
def test_one_hot_returns_row(g, path):
    from tests.gpu_util import DbHandle, to_dev, to_host
    _skip_unbuilt(g, PATHS[path])
    primes = synth.PRIMES_28
    B, D0, D1, L, N = 4, 50, 12, 2, 256
    db = synth.db_tensor(5, D0, D1, L, N, primes)
    istars = [0, 49, 17, 17]
    ct = np.zeros((B, D0, 2, L, N), dtype=np.uint32)
    for c, i in enumerate(istars):
        ct[c, i] = 1
    h = DbHandle(g, db, N, primes, path_mask=PATHS[path])
    try:
        got = to_host(h.rowsel(to_dev(ct), B, PATHS[path]))
    finally:
        h.close()
    for c, i in enumerate(istars):
        for r in range(2):
            assert np.array_equal(got[c, :, r], db[i])


def _sampled_full_size(g, name, path, n_slots=6, variant=None):
    """Full-size workload generated on the device; oracle on sampled slots
    (`variant`: a tile variant to force, else the library's choice)."""
    import torch
    from tests.gpu_util import to_host
    _skip_unbuilt(g, path)
    cfg = synth.config_shapes(name)
    N, L, D0, D1, seed, primes = cfg["N"], cfg["L"], cfg["D0"], cfg["D1"], cfg["seed"], cfg["primes"]
    B = cfg["B"] if isinstance(cfg["B"], int) else max(cfg["B"])
    params = g.gpir_params_create(N, list(primes))
    db_d = torch.empty(D0 * D1 * L * N, dtype=torch.int32, device="cuda")
    g.gpir_fill_uniform(db_d, db_d.numel(), 0, seed, synth.TAG_DB, params, N)
    ct_d = torch.empty(B * D0 * 2 * L * N, dtype=torch.int32, device="cuda")
    g.gpir_fill_uniform(ct_d, ct_d.numel(), 0, seed, synth.TAG_CT, params, N)
    h = g.gpir_db_upload(params, D0, D1, db_d, True, path)
    del db_d
    out = torch.full((B, D1, 2, L, N), -1, dtype=torch.int32, device="cuda")
    try:
        if variant is not None:
            g.gpir_set_variant(h, B, path, variant)
        g.gpir_rowsel_batch(h, B, ct_d, out, path)
        torch.cuda.synchronize()
        g.gpir_sync(None, 60000)
        rng = np.random.default_rng(123)
        slots = [(0, 0), (L - 1, N - 1)] + [(int(rng.integers(0, L)), int(rng.integers(0, N)))
                                            for _ in range(n_slots - 2)]
        ct_s = synth.ct_slots(seed, B, D0, L, N, primes, slots)        # [B][D0][2][S]
        db_s = synth.db_slots(seed, D0, D1, L, N, primes, slots)       # [D0][D1][S]
        got_all = out.view(B, D1, 2, L, N)
        for k, (l, t) in enumerate(slots):
            want = oracle.rowsel(ct_s[:, :, :, None, k:k + 1], db_s[:, :, None, k:k + 1], [primes[l]])
            got = to_host(got_all[:, :, :, l, t].contiguous())
            assert np.array_equal(got, want[:, :, :, 0, 0]), (l, t)
    finally:
        g.gpir_db_free(h)
        g.gpir_params_destroy(params)


@pytest.mark.parametrize("path", PATH_LIST)
def test_full_size_rowsel_32_clients_sampled(g, path):
    _sampled_full_size(g, "c2_rowsel", PATHS[path])


@pytest.mark.parametrize("path", PATH_LIST)
def test_full_size_large_db_sampled(g, path):
    _sampled_full_size(g, "c4_large", PATHS[path], n_slots=4)


def test_device_generator_matches_host(g):
    import torch
    from tests.gpu_util import to_host
    primes = synth.PRIMES_28
    B, D0, L, N = 3, 7, 2, 64
    params = g.gpir_params_create(N, list(primes))
    t = torch.empty(B * D0 * 2 * L * N, dtype=torch.int32, device="cuda")
    g.gpir_fill_uniform(t, t.numel(), 0, 11, synth.TAG_CT, params, N)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(t).reshape(B, D0, 2, L, N), synth.ct_tensor(11, B, D0, L, N, primes))
    # offset start (chunked generation)
    t2 = torch.empty(100, dtype=torch.int32, device="cuda")
    g.gpir_fill_uniform(t2, 100, 500, 11, synth.TAG_CT, params, N)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(t2), synth.ct_tensor(11, B, D0, L, N, primes).ravel()[500:600])
    g.gpir_params_destroy(params)


def test_host_entry_point_matches_device(g):
    import torch
    from tests.gpu_util import DbHandle, to_dev, to_host, make_problem
    primes = synth.PRIMES_28
    B, D0, D1, L, N = 4, 37, 21, 2, 128
    ct, db = make_problem(31, B, D0, D1, L, N, primes)
    want = oracle.rowsel(ct, db, list(primes))
    h = DbHandle(g, db, N, primes, path_mask=1, on_device=False)
    try:
        out = np.zeros((B, D1, 2, L, N), dtype=np.uint32)
        g.gpir_rowsel_batch_host(h.h, B, np.ascontiguousarray(ct), out, 1)
        g.gpir_sync(None, 20000)
        assert np.array_equal(out, want)
        # twice in a row, larger batch grows the workspace
        ct2, _ = make_problem(32, 2 * B, D0, D1, L, N, primes)
        out2 = np.zeros((2 * B, D1, 2, L, N), dtype=np.uint32)
        g.gpir_rowsel_batch_host(h.h, 2 * B, np.ascontiguousarray(ct2), out2, 1)
        g.gpir_sync(None, 20000)
        assert np.array_equal(out2, oracle.rowsel(ct2, db, list(primes)))
    finally:
        h.close()


def test_host_entry_point_chunked_pipeline(g):
    """Batches of 16 or more go through the chunked copy pipeline (uploads,
    RowSel and downloads overlapped over three streams): uneven chunks, pinned
    and pageable buffers, every path, two calls back to back without a sync."""
    import torch
    from tests.gpu_util import DbHandle, make_problem
    primes = synth.PRIMES_28
    B, D0, D1, L, N = 19, 37, 21, 2, 128
    ct, db = make_problem(41, B, D0, D1, L, N, primes)
    ct2, _ = make_problem(42, B, D0, D1, L, N, primes)
    want, want2 = oracle.rowsel(ct, db, list(primes)), oracle.rowsel(ct2, db, list(primes))
    h = DbHandle(g, db, N, primes, path_mask=0)
    try:
        for path in [p for p in (0, 1, 2, 4) if p == 0 or g.gpir_num_variants(p) > 0]:
            ct_p = torch.from_numpy(ct.view(np.int32).copy()).pin_memory()
            ct2_p = torch.from_numpy(ct2.view(np.int32).copy()).pin_memory()
            out_p = torch.full((B, D1, 2, L, N), -1, dtype=torch.int32).pin_memory()
            out2_np = np.zeros((B, D1, 2, L, N), dtype=np.uint32)
            g.gpir_rowsel_batch_host(h.h, B, ct_p, out_p, path)
            g.gpir_rowsel_batch_host(h.h, B, np.ascontiguousarray(ct2), out2_np, path)
            g.gpir_sync(None, 20000)
            assert np.array_equal(out_p.numpy().view(np.uint32), want), "path %d, pinned" % path
            assert np.array_equal(out2_np, want2), "path %d, pageable" % path
    finally:
        h.close()


def test_upload_rejects_out_of_range_residue(g):
    import torch
    from tests.gpu_util import to_dev
    primes = synth.PRIMES_28
    db = synth.db_tensor(3, 4, 4, 2, 32, primes)
    db[2, 1, 1, 7] = primes[1]          # == q1: not canonical
    params = g.gpir_params_create(32, list(primes))
    with pytest.raises(g.GpirError) as ei:
        g.gpir_db_upload(params, 4, 4, to_dev(db), True, 0)
    assert ei.value.code == g.GPIR_ERANGE
    db[2, 1, 1, 7] = primes[0] - 1      # < q0 but it sits in limb 1 where q1 < q0
    with pytest.raises(g.GpirError) as ei:
        g.gpir_db_upload(params, 4, 4, to_dev(db), True, 0)
    assert ei.value.code == g.GPIR_ERANGE
    g.gpir_params_destroy(params)


def test_argument_errors(g):
    import torch
    from tests.gpu_util import DbHandle, to_dev, make_problem
    primes = synth.PRIMES_28
    ct, db = make_problem(1, 2, 8, 8, 2, 32, primes)
    h = DbHandle(g, db, 32, primes, path_mask=1)
    try:
        ct_d = to_dev(ct)
        with pytest.raises(g.GpirError) as ei:     # output overlaps input
            g.gpir_rowsel_batch(h.h, 2, ct_d, ct_d, 1)
        assert ei.value.code == g.GPIR_EINVAL
        out = torch.empty(2 * 8 * 2 * 2 * 32, dtype=torch.int32, device="cuda")
        with pytest.raises(g.GpirError) as ei:     # path not prepared at upload
            g.gpir_rowsel_batch(h.h, 2, ct_d, out, 4)
        assert ei.value.code == g.GPIR_ENOTSUP
        with pytest.raises(g.GpirError) as ei:     # batch 0
            g.gpir_rowsel_batch(h.h, 0, ct_d, out, 1)
        assert ei.value.code == g.GPIR_EINVAL
    finally:
        h.close()


@pytest.mark.parametrize("B", [1, 12])
def test_auto_path_after_autotune(g, B):
    """GPIR_PATH_AUTO after tuning every prepared path: valid choice, same bits."""
    from tests.gpu_util import DbHandle, to_dev, to_host, make_problem
    primes = synth.PRIMES_28
    D0, D1, L, N = 70, 40, 2, 128
    ct, db = make_problem(600 + B, B, D0, D1, L, N, primes)
    want = oracle.rowsel(ct, db, list(primes))
    h = DbHandle(g, db, N, primes, path_mask=0)
    try:
        import torch
        ct_d = to_dev(ct)
        out = torch.full((B, D1, 2, L, N), -1, dtype=torch.int32, device="cuda")
        g.gpir_autotune(h.h, B, ct_d, out, 0)
        assert g.gpir_selected_path(h.h, B) in (1, 2, 4)
        got = to_host(h.rowsel(ct_d, B, 0))
        assert np.array_equal(got, want)
    finally:
        h.close()


def test_debug_checks_reject_non_canonical_ciphertexts(g):
    """With the debug checks on, every RowSel entry point refuses a ciphertext
    residue that is not below its limb's prime (GPIR_ERANGE, nothing computed)
    and still computes canonical inputs bit-exactly; with them off the
    precondition is not checked."""
    import torch
    from tests.gpu_util import DbHandle, to_dev, to_host, make_problem
    primes = synth.PRIMES_28
    B, D0, D1, L, N = 3, 40, 24, 2, 64
    ct, db = make_problem(91, B, D0, D1, L, N, primes)
    want = oracle.rowsel(ct, db, list(primes))
    bad = ct.copy()
    bad[1, 7, 1, 1, 5] = primes[1]          # equal to q1, in limb 1
    h = DbHandle(g, db, N, primes, path_mask=0)
    prev = g.gpir_set_debug(True)
    try:
        for path in [p for p in (1, 2, 4) if g.gpir_num_variants(p) > 0]:
            assert np.array_equal(to_host(h.rowsel(to_dev(ct), B, path)), want), path
            with pytest.raises(g.GpirError) as ei:
                h.rowsel(to_dev(bad), B, path)
            assert ei.value.code == g.GPIR_ERANGE, path
        out = torch.empty((B, D1, 2, L, N), dtype=torch.int32, device="cuda")
        with pytest.raises(g.GpirError) as ei:
            g.gpir_rowsel_multi([(h.h, B, to_dev(bad), out)], 0)
        assert ei.value.code == g.GPIR_ERANGE
        if g.gpir_num_variants(4) > 0:
            with pytest.raises(g.GpirError) as ei:
                g.gpir_rowsel_batch_noalloc(h.h, B, to_dev(bad), out)
            assert ei.value.code == g.GPIR_ERANGE
        out_h = np.zeros((B, D1, 2, L, N), dtype=np.uint32)
        with pytest.raises(g.GpirError) as ei:
            g.gpir_rowsel_batch_host(h.h, B, np.ascontiguousarray(bad), out_h, 1)
        assert ei.value.code == g.GPIR_ERANGE
    finally:
        g.gpir_set_debug(prev)
    h.rowsel(to_dev(bad), B, 1)              # off: accepted (the result is unspecified)
    h.close()


@pytest.mark.parametrize("path", PATH_LIST)
def test_largest_ring_degree(g, path):
    """The largest ring degree the ABI accepts, N = 2^16, with the two largest
    primes = 1 mod 2^17 below 2^28, two limbs, every path (the smallest, N = 4,
    is in SHAPES)."""
    _check_full(g, 3, 20, 9, 2, 65536, (268042241, 265420801), 500, PATHS[path])
