"""Repository rules checked on the CPU: the product path never reaches the CPU
oracle or the git-ignored scratch directory, every GPU test module is marked,
and no committed source names the batched-copy CUDA calls this project does
not use (one cudaMemcpyAsync per copy instead)."""

import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2604_04696_gb300")


def _ignored_dirs():
    """Directory entries of .gitignore (lines ending in '/'), without slashes."""
    try:
        lines = open(os.path.join(ROOT, ".gitignore"), encoding="utf-8").read().splitlines()
    except OSError:
        return set()
    return {ln.strip().strip("/") for ln in lines if ln.strip().endswith("/") and not ln.startswith("#")}


def _committed_files():
    r = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True)
    if r.returncode != 0:
        # no git metadata (a copy of the tree): everything but hidden and ignored directories
        skip = _ignored_dirs()
        files = []
        for d, dirs, fs in os.walk(ROOT):
            rel = os.path.relpath(d, ROOT)
            dirs[:] = [x for x in dirs if not x.startswith(".") and x not in skip
                       and os.path.join(rel, x).lstrip("./") not in skip]
            files += [os.path.relpath(os.path.join(d, f), ROOT) for f in fs]
        return files
    return [f for f in r.stdout.splitlines() if f]


def test_product_package_never_imports_the_oracle_or_scratch():
    imp = re.compile(r"^\s*(import\s+oracle\b|from\s+oracle\b|from\s+\.\.?\s*import\s+oracle\b)", re.M)
    scratch = re.compile(r"""["'/\\]_work["'/\\]""")
    for d, _, fs in os.walk(PKG):
        for f in fs:
            if not f.endswith((".py", ".cu", ".cuh", ".h")):
                continue
            src = open(os.path.join(d, f), encoding="utf-8").read()
            assert not imp.search(src), os.path.join(d, f)
            assert not scratch.search(src), os.path.join(d, f)


def test_gpu_test_modules_are_marked():
    for f in os.listdir(os.path.join(ROOT, "tests")):
        if f.startswith("test_") and f.endswith(".py"):
            src = open(os.path.join(ROOT, "tests", f), encoding="utf-8").read()
            uses_gpu = "gpu_util.lib()" in src or 'device="cuda"' in src
            if uses_gpu:
                assert re.search(r"^pytestmark\s*=\s*pytest\.mark\.gpu", src, re.M) or "@pytest.mark.gpu" in src, f


def test_no_batched_copy_calls_named():
    names = [p + "Memcpy" + s + "BatchAsync" for p in ("cuda", "cu") for s in ("", "3D")]
    for f in _committed_files():
        if f.endswith(".md") or not os.path.isfile(os.path.join(ROOT, f)):
            continue
        try:
            src = open(os.path.join(ROOT, f), encoding="utf-8", errors="ignore").read()
        except OSError:
            continue
        for n in names:
            assert n not in src, (f, n)
