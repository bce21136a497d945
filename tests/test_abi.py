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


C_CALLER = r"""
#include "pmp.h"
#include <stdio.h>

int main(void)
{
    if (pmp_gathered_rows(PMP_KIND_FEEDBACK) != 12 || pmp_gathered_rows(PMP_KIND_SINK) != 8) return 2;
    pmp_params p = {0};
    p.kind = PMP_KIND_FEEDBACK;
    p.subsample = 4;
    p.r_K = 0.5; /* below the allowed range: rejected before any device work */
    p.gamma = 5.0 / 3.0;
    p.A_sf = 30.0;
    p.A_p = 5.0;
    p.mu_H = 1.0;
    p.RM_ej = 0.027;
    p.RM_st = 1.0;
    p.eps_K = 0.28;
    pmp_ctx *ctx = (pmp_ctx *)&p; /* must come back NULL */
    if (pmp_create(&ctx, &p, NULL) != PMP_ERR_ARG || ctx != NULL) return 3;
    pmp_destroy(NULL);
    puts("ok");
    return 0;
}
"""


def test_header_compiles_as_c_and_the_library_links_from_c(lib, tmp_path):
    """A caller written in C11 (no C++, no Python) includes only pmp.h, links
    libpmp.so and makes calls that need no GPU."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    import subprocess

    src = tmp_path / "caller.c"
    src.write_text(C_CALLER)
    libdir = os.path.dirname(lib._name)
    exe = tmp_path / "caller"
    subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-L", libdir, "-lpmp", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)


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
