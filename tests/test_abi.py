"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function include/pmp.h declares.  No compute calls (no GPU needed)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "pmp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pmp_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2509_18261_gb300 import build

    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared()
    for n in ("pmp_gather", "pmp_deposit", "pmp_fold_ghosts", "pmp_apply_limited", "pmp_backward"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export():
    from paper_2509_18261_gb300 import pmp

    assert sorted(pmp.EXPORTS) == declared()


def test_gathered_rows_without_gpu(lib):
    lib.pmp_gathered_rows.restype = ctypes.c_int32
    assert lib.pmp_gathered_rows(0) == 12 and lib.pmp_gathered_rows(1) == 8 and lib.pmp_gathered_rows(7) == 0


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    """No CPU fallback: with libpmp.so absent, the first call raises instead
    of computing anything another way."""
    from paper_2509_18261_gb300 import pmp

    monkeypatch.setattr(pmp, "_lib", None)
    monkeypatch.setattr(pmp, "LIB_PATH", str(tmp_path / "libpmp.so"))
    with pytest.raises(RuntimeError, match="libpmp.so not found"):
        pmp.load()
    with pytest.raises(RuntimeError):
        pmp.pmp_gathered_rows(0)
