"""The C-ABI library loads and exports every entry point include/bk.h declares.

No compute call is made here (no GPU needed): only symbol lookup and the two entry
points that touch no device (bk_default_opts, bk_status_string)."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bk.h")
LIB = os.path.join(ROOT, "paper_2501_18717_gb300", "libbk.so")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bk_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        r = subprocess.run([sys.executable, "-m", "paper_2501_18717_gb300.build"], cwd=ROOT, capture_output=True,
                           text=True)
        if r.returncode != 0:
            pytest.skip("nvcc build failed: " + r.stderr[-500:])
    return ctypes.CDLL(LIB)


def test_header_declares_entry_points():
    names = declared()
    for n in ["bk_create", "bk_destroy", "bk_solve", "bk_block_apply", "bk_gram", "bk_chol_solve", "bk_gaussian"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points(lib):
    from paper_2501_18717_gb300 import bk
    o = bk.default_opts()
    assert o.tol == 1e-10 and o.sketch == 20 and o.inner == bk.BK_PREC_FP64 and o.check_every == 8
    assert bk.status_string(bk.BK_BREAKDOWN).startswith("block breakdown")
    assert set(bk.EXPORTS) <= set(declared())


NULL_CTX_PROBE = r"""
import ctypes, sys
sys.path.insert(0, sys.argv[1])
from paper_2501_18717_gb300 import bk
L = bk._lib
o, info = bk.default_opts(), bk.Info()
op = bk.Operator(bk.BK_DENSE, bk.BK_F64, 4, 4, 4, None, None, None, 0)
buf = (ctypes.c_double * 64)()
p = ctypes.cast(buf, ctypes.c_void_p)
mu = (ctypes.c_double * 2)(0.1, 0.2)
pm = ctypes.cast(mu, ctypes.c_void_p)
A, O, I = ctypes.byref(op), ctypes.byref(o), ctypes.byref(info)
calls = {
    "bk_solve": lambda: L.bk_solve(None, A, 0.0, p, p, O, I),
    "bk_ridge_path": lambda: L.bk_ridge_path(None, A, 2, pm, p, p, O, I),
    "bk_sample": lambda: L.bk_sample(None, A, 0.0, 1, p, p, 8, O, I),
    "bk_sample_isqrt": lambda: L.bk_sample_isqrt(None, A, 0.0, 1, p, p, 8, O, I),
    "bk_nystrom_pcg": lambda: L.bk_nystrom_pcg(None, A, 0.0, p, p, 1, O, I),
    "bk_solve_shrink": lambda: L.bk_solve_shrink(None, A, 0.0, p, p, 1, O, I),
    "bk_block_apply": lambda: L.bk_block_apply(None, A, 0.0, bk.BK_F64, 1, p, p, 4, p),
    "bk_gram": lambda: L.bk_gram(None, bk.BK_F64, 4, 1, p, p, 4, p),
    "bk_chol_solve": lambda: L.bk_chol_solve(None, 2, p, p, p),
    "bk_gaussian": lambda: L.bk_gaussian(None, 1, 3, 4, 0, p),
    "bk_solve_batched": lambda: L.bk_solve_batched(None, 1, A, pm, p, p, O, None),
    "bk_autotune": lambda: L.bk_autotune(None, 1, A, pm, p, p, 1, O, None),
}
for k, f in calls.items():
    print(k, f())
"""


def test_null_context_is_an_argument_error(lib):
    """Every entry point that needs a context returns BK_ERR_ARG for a null one, before
    any device work (so this runs without a GPU). Run in a child process: a crash
    there fails the test instead of the session."""
    from paper_2501_18717_gb300 import bk
    r = subprocess.run([sys.executable, "-c", NULL_CTX_PROBE, ROOT], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    got = dict(line.split() for line in r.stdout.strip().splitlines())
    assert len(got) == 12
    assert all(int(v) == bk.BK_ERR_ARG for v in got.values()), got
