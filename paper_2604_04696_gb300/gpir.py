"""Thin ctypes binding of libgpir.so: the C ABI of include/gpir.h, same names.

Argument marshalling only: every step of RowSel runs in the library's CUDA
kernels. Device buffers may be passed as integers (device addresses) or as
objects with a ``data_ptr()`` method (torch tensors); streams as integers
(cudaStream_t) or objects with a ``cuda_stream`` attribute. There is no CPU
fallback: if the library cannot be loaded, importing this module raises.
"""

import ctypes
import os

from . import _build

GPIR_OK = 0
GPIR_EINVAL = -1
GPIR_ERANGE = -2
GPIR_ENOMEM = -3
GPIR_ECUDA = -4
GPIR_ETIMEOUT = -5
GPIR_ENOTSUP = -6
GPIR_ETOOBIG = -7
GPIR_NOALLOC_SCRATCH_BYTES = 64 << 20

GPIR_PATH_AUTO = 0
GPIR_PATH_CUDACORE = 1
GPIR_PATH_IMMA = 2
GPIR_PATH_TC = 4
GPIR_PATH_ALL = 7

GPIR_MAX_LIMBS = 8
GPIR_MIN_N = 4
GPIR_MAX_N = 65536
GPIR_MAX_PRIME_BITS = 28
GPIR_MAX_BATCH = 1 << 30


class GpirError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s failed: %s (%d)%s" % (what, _strerror(code), code, _cuda_detail(code)))


class gpir_trace_record_t(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("ms", ctypes.c_float)]


class gpir_job_t(ctypes.Structure):
    _fields_ = [("db", ctypes.c_void_p), ("batch", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("ct", ctypes.c_void_p), ("out", ctypes.c_void_p)]


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libgpir.so is not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    P, U32, U64, I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    sig = {
        "gpir_params_create": (I, [U32, U32, ctypes.POINTER(U32), ctypes.POINTER(P)]),
        "gpir_params_destroy": (I, [P]),
        "gpir_db_upload": (I, [P, U32, U32, P, I, U32, P, ctypes.POINTER(P)]),
        "gpir_db_free": (I, [P]),
        "gpir_db_device_bytes": (ctypes.c_size_t, [P]),
        "gpir_rowsel_batch": (I, [P, U32, P, P, I, P]),
        "gpir_rowsel_batch_host": (I, [P, U32, P, P, I, P]),
        "gpir_rowsel_multi": (I, [ctypes.POINTER(gpir_job_t), U32, I, P]),
        "gpir_rowsel_batch_noalloc": (I, [P, U32, P, P, P]),
        "gpir_coltor": (I, [P, U32, U32, P, P, P, P]),
        "gpir_coltor_gadget_digits": (I, [P]),
        "gpir_expand_query": (I, [P, U32, U32, U32, P, P, P, P]),
        "gpir_pir_batch": (I, [P, U32, U32, P, P, P, P, P, P, I, P]),
        "gpir_graph_create": (I, [ctypes.POINTER(gpir_job_t), U32, I, P, ctypes.POINTER(P)]),
        "gpir_graph_launch": (I, [P, P]),
        "gpir_graph_destroy": (I, [P]),
        "gpir_sync": (I, [P, U32]),
        "gpir_selftest_bounded_wait": (I, [P]),
        "gpir_set_debug": (I, [I]),
        "gpir_set_fail_alloc": (ctypes.c_long, [ctypes.c_long]),
        "gpir_autotune": (I, [P, U32, P, P, I, P, ctypes.POINTER(I)]),
        "gpir_num_variants": (I, [I]),
        "gpir_selected_variant": (I, [P, U32, I]),
        "gpir_selected_path": (I, [P, U32]),
        "gpir_set_variant": (I, [P, U32, I, I]),
        "gpir_fill_uniform": (I, [P, U64, U64, U64, U64, P, U64, P]),
        "gpir_trace_enable": (I, [I]),
        "gpir_trace_read": (I, [ctypes.POINTER(gpir_trace_record_t), U32, ctypes.POINTER(U32)]),
        "gpir_trace_counters": (I, [ctypes.POINTER(ctypes.c_ulonglong), U32, ctypes.POINTER(U32)]),
        "gpir_strerror": (ctypes.c_char_p, [I]),
        "gpir_last_cuda_error": (ctypes.c_char_p, []),
        "gpir_version": (I, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def _strerror(code):
    return lib.gpir_strerror(code).decode()


def _cuda_detail(code):
    if code in (GPIR_ECUDA, GPIR_ENOMEM):
        return ": " + lib.gpir_last_cuda_error().decode()
    return ""


def _check(rc, what):
    if rc != GPIR_OK:
        raise GpirError(rc, what)
    return rc


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):          # numpy array (host)
        return x.ctypes.data
    return int(x)


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


def gpir_params_create(n, primes):
    arr = (ctypes.c_uint32 * len(primes))(*[int(q) for q in primes])
    h = ctypes.c_void_p()
    _check(lib.gpir_params_create(int(n), len(primes), arr, ctypes.byref(h)), "gpir_params_create")
    return h


def gpir_params_destroy(params):
    return lib.gpir_params_destroy(params)


def gpir_db_upload(params, d0, d1, db_ntt, on_device, path_mask=0, stream=None):
    h = ctypes.c_void_p()
    _check(lib.gpir_db_upload(params, int(d0), int(d1), _ptr(db_ntt), 1 if on_device else 0, int(path_mask),
                              _stream(stream), ctypes.byref(h)), "gpir_db_upload")
    return h


def gpir_db_free(db):
    return lib.gpir_db_free(db)


def gpir_db_device_bytes(db):
    return lib.gpir_db_device_bytes(db)


def gpir_rowsel_batch(db, batch, ct_dev, out_dev, path=GPIR_PATH_AUTO, stream=None):
    return _check(lib.gpir_rowsel_batch(db, int(batch), _ptr(ct_dev), _ptr(out_dev), int(path), _stream(stream)),
                  "gpir_rowsel_batch")


def gpir_rowsel_batch_host(db, batch, ct_host, out_host, path=GPIR_PATH_AUTO, stream=None):
    return _check(lib.gpir_rowsel_batch_host(db, int(batch), _ptr(ct_host), _ptr(out_host), int(path),
                                             _stream(stream)), "gpir_rowsel_batch_host")


def gpir_rowsel_batch_noalloc(db, batch, ct_dev, out_dev, stream=None):
    """Tensor-core RowSel with no device allocation (fixed internal workspace)."""
    return _check(lib.gpir_rowsel_batch_noalloc(db, int(batch), _ptr(ct_dev), _ptr(out_dev), _stream(stream)),
                  "gpir_rowsel_batch_noalloc")


def gpir_rowsel_multi(jobs, path=GPIR_PATH_AUTO, stream=None):
    """jobs: sequence of (db_handle, batch, ct_dev, out_dev)."""
    return _check(lib.gpir_rowsel_multi(_jobs(jobs), len(jobs), int(path), _stream(stream)), "gpir_rowsel_multi")


def _jobs(jobs):
    arr = (gpir_job_t * len(jobs))()
    for k, (db, batch, ct, out) in enumerate(jobs):
        arr[k].db = db.value if isinstance(db, ctypes.c_void_p) else db
        arr[k].batch = int(batch)
        arr[k].ct = _ptr(ct)
        arr[k].out = _ptr(out)
    return arr


def gpir_graph_create(jobs, path=GPIR_PATH_AUTO, stream=None):
    """Capture one gpir_rowsel_multi call over `jobs` into a CUDA graph."""
    h = ctypes.c_void_p()
    _check(lib.gpir_graph_create(_jobs(jobs), len(jobs), int(path), _stream(stream), ctypes.byref(h)),
           "gpir_graph_create")
    return h


def gpir_graph_launch(graph, stream=None):
    return _check(lib.gpir_graph_launch(graph, _stream(stream)), "gpir_graph_launch")


def gpir_graph_destroy(graph):
    return lib.gpir_graph_destroy(graph)


def gpir_sync(stream=None, timeout_ms=0):
    return _check(lib.gpir_sync(_stream(stream), int(timeout_ms)), "gpir_sync")


def gpir_set_debug(on=True):
    """Debug checks of the ciphertext residues on or off; returns the previous setting."""
    return lib.gpir_set_debug(1 if on else 0)


def gpir_set_fail_alloc(n):
    """Arm (n > 0: the n-th device allocation from now fails) or disarm (n <= 0)
    the allocation-failure injection; returns the previous countdown."""
    return lib.gpir_set_fail_alloc(int(n))


def gpir_selftest_bounded_wait(stream=None):
    return _check(lib.gpir_selftest_bounded_wait(_stream(stream)), "gpir_selftest_bounded_wait")


def gpir_sync_rc(stream=None, timeout_ms=0):
    """gpir_sync returning the raw code instead of raising."""
    return lib.gpir_sync(_stream(stream), int(timeout_ms))


def gpir_autotune(db, batch, ct_dev, out_dev, path, stream=None):
    v = ctypes.c_int(-1)
    _check(lib.gpir_autotune(db, int(batch), _ptr(ct_dev), _ptr(out_dev), int(path), _stream(stream),
                             ctypes.byref(v)), "gpir_autotune")
    return v.value


def gpir_coltor(params, batch, d1, ct_dev, rgsw_dev, out_dev, stream=None):
    return _check(lib.gpir_coltor(params, int(batch), int(d1), _ptr(ct_dev), _ptr(rgsw_dev), _ptr(out_dev),
                                  _stream(stream)), "gpir_coltor")


def gpir_expand_query(params, batch, stages, n_out, query_dev, evk_dev, out_dev, stream=None):
    return _check(lib.gpir_expand_query(params, int(batch), int(stages), int(n_out), _ptr(query_dev),
                                        _ptr(evk_dev), _ptr(out_dev),
                                        _stream(stream)), "gpir_expand_query")


def gpir_pir_batch(db, batch, stages, query_dev, evk_dev, rgsw_dev, sel_dev, rows_dev, out_dev, path=0, stream=None):
    return _check(lib.gpir_pir_batch(db, int(batch), int(stages), _ptr(query_dev), _ptr(evk_dev), _ptr(rgsw_dev),
                                     _ptr(sel_dev), _ptr(rows_dev), _ptr(out_dev), int(path), _stream(stream)),
                  "gpir_pir_batch")


def gpir_coltor_gadget_digits(params):
    r = lib.gpir_coltor_gadget_digits(params)
    if r < 0:
        _check(r, "gpir_coltor_gadget_digits")
    return r


def gpir_num_variants(path):
    return lib.gpir_num_variants(int(path))


def gpir_selected_variant(db, batch, path):
    return lib.gpir_selected_variant(db, int(batch), int(path))


def gpir_selected_path(db, batch):
    return lib.gpir_selected_path(db, int(batch))


def gpir_set_variant(db, batch, path, variant):
    return _check(lib.gpir_set_variant(db, int(batch), int(path), int(variant)), "gpir_set_variant")


def gpir_fill_uniform(dst_dev, count, start, seed, tag, params, inner, stream=None):
    return _check(lib.gpir_fill_uniform(_ptr(dst_dev), int(count), int(start), int(seed), int(tag), params,
                                        int(inner), _stream(stream)), "gpir_fill_uniform")


def gpir_trace_enable(on=True, counters=False):
    """on: per-launch CUDA-event times; counters: also the role-counting
    kernel instantiations (level 2, slower)."""
    return _check(lib.gpir_trace_enable((2 if counters else 1) if on else 0), "gpir_trace_enable")


def gpir_trace_read(max_records=4096):
    """[(kernel name, device ms)] of the launches since the last read (waits for them)."""
    buf = (gpir_trace_record_t * max_records)()
    n = ctypes.c_uint32(0)
    _check(lib.gpir_trace_read(buf, max_records, ctypes.byref(n)), "gpir_trace_read")
    return [(buf[i].name.decode(), float(buf[i].ms)) for i in range(n.value)]


FUSED_COUNTERS = ["producer_wait_ready", "producer_wait_empty", "mma_wait_full", "mma_wait_acc_empty",
                  "epilogue_wait_acc_full", "epilogue_wait_stage", "ingest_wait_consumed", "ingest_wait_box",
                  "ingest_busy", "ingest_wait_slabs", "ingest_push", "cta_cycles"]


TMEM_COUNTERS = ["p_wait_ready", "p_wait_empty", "c_wait_full", "c_busy", "c_store", "m_wait_a", "m_wait_acc", "m_issue",
                 "m_handoff", "e_wait_acc", "e_busy", "i_wait_slot", "i_wait_box", "i_busy", "i_fence", "cta_cycles"]


def gpir_trace_counters(names=None):
    """{name: cycles} of the last traced fused, cluster or tensor-memory launch
    (names: FUSED_COUNTERS, the default, or TMEM_COUNTERS)."""
    names = FUSED_COUNTERS if names is None else names
    buf = (ctypes.c_ulonglong * 32)()
    n = ctypes.c_uint32(0)
    _check(lib.gpir_trace_counters(buf, 32, ctypes.byref(n)), "gpir_trace_counters")
    return {names[i] if i < len(names) else str(i): int(buf[i]) for i in range(n.value)}


def gpir_strerror(code):
    return _strerror(code)


def gpir_version():
    return lib.gpir_version()
