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
