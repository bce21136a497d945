"""The library's correctly rounded FP64 quotient and square root from integer
and FP32 instructions (pmp_exact.cuh, used by the kernels for the divisions
and square roots of Eq. du and the sink formulas), and its comparisons with
0 and 1 decided on the bit patterns.  A binary64 quotient or
square root rounded to nearest is unique, so the check is bit equality:

- on the host, the header compiled by g++ against the C library's sqrt and
  the host's IEEE division (tests/native/exact_harness.cpp: random operands
  over the normal range, squares and products perturbed by a few units in the
  last place, exact squares and quotients, significand extremes, exponents at
  the edges of the fast path);
- on the GPU, pmp_exact_math against the device's own sqrt and division
  (torch), and against numpy on the host for a sample, special operands
  included.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2509_18261_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    out = str(tmp_path_factory.mktemp("exact") / "exact_harness.so")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                           "-I", CSRC, os.path.join(HERE, "native", "exact_harness.cpp"), "-o", out])
    lib = ctypes.CDLL(out)
    lib.exact_check.argtypes = [ctypes.c_uint64, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong),
                                ctypes.POINTER(ctypes.c_double)]
    lib.exact_check_compare.argtypes = [ctypes.c_uint64, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double)]
    lib.exact_check_compare.restype = ctypes.c_longlong
    lib.exact_check_half_odd.argtypes = [ctypes.c_longlong, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]
    lib.exact_check_half_odd.restype = ctypes.c_longlong
    return lib


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_host_build_matches_the_c_library(harness, seed):
    counts = (ctypes.c_longlong * 4)()
    bad = (ctypes.c_double * 3)()
    harness.exact_check(seed, 10_000_000, counts, bad)
    assert counts[0] == counts[2] == 10_000_000
    assert counts[1] == 0, f"sqrt wrong for x = {bad[0]!r}"
    assert counts[3] == 0, f"quotient wrong for {bad[1]!r} / {bad[2]!r}"


def test_host_bit_pattern_comparisons_match_ieee(harness):
    """x > 0, x >= 0, x < 0, x != 0, x > 1 and x < 1 decided on the bits
    (used by the Eq. lambda limiter) against the IEEE comparisons."""
    bad = ctypes.c_double()
    assert harness.exact_check_compare(7, 2_000_000, ctypes.byref(bad)) == 0, f"comparison wrong for {bad.value!r}"


def test_host_cell_centre_from_bits_matches_the_conversion(harness):
    """c + 1/2 built from the bits of 2c + 1 (the deposit's offset table)
    against (double)c + 0.5, for every cell index of boxes up to 2^22 cells
    per axis and the ends of the int range."""
    bad = ctypes.c_longlong()
    assert harness.exact_check_half_odd(-(1 << 22), 1 << 22, ctypes.byref(bad)) == 0, f"wrong for c = {bad.value}"
    assert harness.exact_check_half_odd(-(1 << 30), -(1 << 30) + 1000, ctypes.byref(bad)) == 0, bad.value
    assert harness.exact_check_half_odd((1 << 30) - 1001, (1 << 30) - 1, ctypes.byref(bad)) == 0, bad.value


def _operands(n, seed):
    """Bit patterns over the whole double range (all exponents, both signs),
    plus squares and products perturbed by a few ulps."""
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 2**63, n, dtype=np.int64).view(np.uint64) | (rng.integers(0, 2, n, dtype=np.uint64) << 63)
    b = rng.integers(0, 2**63, n, dtype=np.int64).view(np.uint64) | (rng.integers(0, 2, n, dtype=np.uint64) << 63)
    a, b = a.view(np.float64), b.view(np.float64)
    m = n // 3
    y = np.exp(rng.uniform(-300, 300, m))
    with np.errstate(all="ignore"):
        sq = (y * y).view(np.int64) + rng.integers(-3, 4, m)
        a[:m] = np.abs(sq.view(np.float64))
        q = np.exp(rng.uniform(-300, 300, m))
        pr = (q * y).view(np.int64) + rng.integers(-3, 4, m)
    a[m:2 * m] = pr.view(np.float64)
    b[m:2 * m] = y
    special = np.array([0.0, -0.0, 5e-324, 2.2250738585072014e-308, 2.225073858507201e-308, 1.7976931348623157e308,
                        np.inf, -np.inf, np.nan, 1.0, -1.0, 2.0, 0.5, 3.0, 1e-300, 1e300])
    k = len(special)
    a[-k * k:] = np.repeat(special, k)
    b[-k * k:] = np.tile(special, k)
    return a, b


def _same(x, y):
    return (x.view(np.uint64) == y.view(np.uint64)) | (np.isnan(x) & np.isnan(y))


@pytest.mark.gpu
def test_device_matches_the_gpu_and_numpy():
    import torch

    from paper_2509_18261_gb300 import pmp

    for seed in range(4):
        a, b = _operands(8_000_000, 100 + seed)
        ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        quot, root = torch.empty_like(ta), torch.empty_like(ta)
        pmp.pmp_exact_math(ta, tb, quot, root)
        want_q, want_r = ta / tb, torch.sqrt(ta)
        torch.cuda.synchronize()
        q, r = quot.cpu().numpy(), root.cpu().numpy()
        wq, wr = want_q.cpu().numpy(), want_r.cpu().numpy()
        assert _same(q, wq).all(), f"quotient: {np.count_nonzero(~_same(q, wq))} differ"
        assert _same(r, wr).all(), f"sqrt: {np.count_nonzero(~_same(r, wr))} differ"
        idx = np.random.default_rng(seed).choice(len(a), 200_000, replace=False)
        idx = np.concatenate([idx, np.arange(len(a) - 256, len(a))])
        with np.errstate(all="ignore"):
            assert _same(q[idx], a[idx] / b[idx]).all()
            assert _same(r[idx], np.sqrt(a[idx])).all()


@pytest.mark.gpu
def test_device_empty_and_bad_arguments():
    import torch

    from paper_2509_18261_gb300 import pmp

    z = torch.empty(0, dtype=torch.float64, device="cuda")
    pmp.pmp_exact_math(z, z, z, z)
    lib = pmp.load()
    assert lib.pmp_exact_math(None, None, 4, None, None, None) == 1  # PMP_ERR_ARG
    assert lib.pmp_exact_math(None, None, -1, None, None, None) == 1  # PMP_ERR_ARG
