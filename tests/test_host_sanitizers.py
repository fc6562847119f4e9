"""The library's host code under AddressSanitizer and UndefinedBehaviorSanitizer
(CPU only, no GPU needed).

Every translation unit is compiled again with the sanitizers on the host side
(device code is unchanged) into a temporary directory, and a child Python with
the sanitizer runtimes preloaded loads that build through the normal binding
and runs the calls that need no GPU: params creation and every params check,
argument validation of every entry point, error strings, the debug switch.
Any sanitizer report, or any call answering differently from the normal
build, fails the test."""

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
sys.path.insert(0, ROOT)
from paper_2604_04696_gb300 import _build
_build.LIB = LIBPATH
_build.build = lambda *a, **k: LIBPATH
from paper_2604_04696_gb300 import gpir as g
import synth
q0, q1 = synth.PRIMES_28
for _ in range(3):
    p = g.gpir_params_create(4096, [q0, q1])
    g.gpir_params_destroy(p)
assert g.gpir_params_create(4, [17, 41]).value
assert g.gpir_params_create(65536, [786433]).value
bad = [(4096, [q0 + 2]), (4096, [q0 + 4096]), (3000, [q0]), (2, [17]), (131072, [q0]),
       (4096, [(1 << 28) + 8193]), (4096, []), (4096, [q0] * 9)]
for n, primes in bad:
    try:
        g.gpir_params_create(n, primes)
    except g.GpirError as e:
        assert e.code == g.GPIR_EINVAL, (n, primes, e.code)
    else:
        raise SystemExit("accepted bad params %r" % ((n, primes),))
for code in range(-12, 2):
    assert g.gpir_strerror(code)
assert g.gpir_version() == 100
assert g.gpir_set_debug(True) in (0, 1)
assert g.gpir_set_debug(False) == 1
L = g.lib
assert L.gpir_rowsel_batch(None, 1, None, None, 0, None) == g.GPIR_EINVAL
assert L.gpir_rowsel_multi(None, 0, 0, None) == g.GPIR_EINVAL
assert L.gpir_db_upload(None, 1, 1, None, 0, 0, None, None) == g.GPIR_EINVAL
assert L.gpir_db_free(None) == g.GPIR_OK
assert L.gpir_params_destroy(None) in (g.GPIR_OK, g.GPIR_EINVAL)
p = g.gpir_params_create(64, [q0, q1])
A, B, C = 1 << 40, 2 << 40, 3 << 40
for d1 in (0, 1, 3, 6):
    assert L.gpir_coltor(p, 1, d1, A, B, C, None) == g.GPIR_EINVAL
assert L.gpir_coltor(p, 1, 4, A, B, A + 64, None) == g.GPIR_EINVAL
assert L.gpir_expand_query(p, 1, 2, 5, A, B, C, None) == g.GPIR_EINVAL
assert L.gpir_expand_query(p, 1, 7, 4, A, B, C, None) == g.GPIR_EINVAL
assert L.gpir_expand_query(p, 1, 2, 4, A, B, A + 64, None) == g.GPIR_EINVAL
assert L.gpir_pir_batch(None, 1, 2, A, B, C, A, B, C, 0, None) == g.GPIR_EINVAL
g.gpir_params_destroy(p)
print("host checks ok")
'''


def _runtime(name):
    try:
        r = subprocess.run(["gcc", "-print-file-name=" + name], capture_output=True, text=True, check=True)
    except (OSError, subprocess.CalledProcessError):
        return None
    path = r.stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


def test_host_code_under_asan_and_ubsan(tmp_path):
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not asan or not ubsan:
        pytest.skip("sanitizer runtimes not installed")
    from paper_2604_04696_gb300 import _build as B
    # one sanitizer per -Xcompiler: nvcc splits its argument at commas
    san = ["-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined",
           "-Xcompiler", "-fno-omit-frame-pointer"]
    nvcc = B._nvcc()

    def compile_one(src):
        obj = str(tmp_path / src.replace(".cu", ".o"))
        cmd = [nvcc] + B.ARCH + B.CFLAGS + san + ["-c", os.path.join(B.CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
        return obj

    with ThreadPoolExecutor(max_workers=min(len(B.SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, B.SOURCES))
    lib = str(tmp_path / "libgpir_san.so")
    r = subprocess.run([nvcc] + B.ARCH + ["-shared", "-o", lib] + objs +
                       ["-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    env = dict(os.environ)
    env["LD_PRELOAD"] = asan + ":" + ubsan
    env["ASAN_OPTIONS"] = "detect_leaks=0:halt_on_error=1"
    env["UBSAN_OPTIONS"] = "halt_on_error=1:print_stacktrace=1"
    env.pop("GPIR_DEBUG", None)
    script = "ROOT = %r\nLIBPATH = %r\n" % (ROOT, lib) + SCRIPT
    r = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True, cwd=ROOT,
                       timeout=300)
    report = r.stderr[-4000:]
    assert r.returncode == 0, report
    assert "AddressSanitizer" not in r.stderr and "runtime error" not in r.stderr, report
    assert r.stdout.strip().endswith("host checks ok"), r.stdout[-1000:]
