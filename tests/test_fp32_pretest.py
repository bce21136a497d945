"""Soundness of the sink limiter's FP32 pre-test (k_sink_eta_apply).

The kernel decides the common case eta = 1 of the accretion limiter
(Sec. 3.1.1) in FP32: a value truncated from FP64 to FP32, cap rounded down,
rho_min rounded up, and a 2^-16 relative margin on each comparison.  It must
never say "eta = 1" where the FP64 tests a <= RN(cap rho) and
a <= RN(rho - rho_min) fail.  numpy's float32 operations are IEEE
round-to-nearest, like the GPU's FP32 pipe without contraction, so the
pre-test restated here runs the same operations; the inputs crowd the two
decision boundaries and the ends of the FP32 range.
"""
import numpy as np

F32 = np.float32


def f32_trunc(v):
    """FP64 -> FP32 by truncating the significand (toward zero); NaN outside the
    FP32 normal range, 0 for +-0 (the kernel's conversion)."""
    v = np.asarray(v, dtype=np.float64)
    bits = v.view(np.uint64)
    hi = (bits >> np.uint64(32)).astype(np.uint64)
    lo = (bits & np.uint64(0xFFFFFFFF)).astype(np.uint64)
    e = ((hi >> np.uint64(20)) & np.uint64(0x7FF)).astype(np.int64) - 1023 + 127
    out = ((hi & np.uint64(0x80000000)) | (np.clip(e, 0, 255).astype(np.uint64) << np.uint64(23))
           | ((hi & np.uint64(0xFFFFF)) << np.uint64(3)) | (lo >> np.uint64(29))).astype(np.uint32)
    res = out.view(np.float32).copy()
    bad = (e <= 0) | (e >= 255)
    zero = (bits << np.uint64(1)) == 0
    res[bad & ~zero] = np.nan
    res[zero] = 0.0
    return res


def round_down_f32(x):
    f = F32(x)
    return np.nextafter(f, F32(0)) if float(f) > x else f


def round_up_f32(x):
    f = F32(x)
    return np.nextafter(f, F32(3e38)) if float(f) < x else f


def pretest(rho, d0, cap_lo, rmin_hi):
    with np.errstate(all="ignore"):
        af = -f32_trunc(d0)
        rf = f32_trunc(rho)
        up = af * F32(1.0000152587890625)
        t1 = (cap_lo * rf) * F32(0.9999847412109375)
        t2 = (rf - rmin_hi) * F32(0.9999847412109375)
        return (up < t1) & (up < t2) & (t1 < F32(1e30))


def exact(rho, a, cap, rho_min):
    return (a <= cap * rho) & (a <= rho - rho_min)


def _check(rho, a, cap, rho_min):
    rho = np.asarray(rho, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    ok = pretest(rho, -a, round_down_f32(cap), round_up_f32(rho_min))
    assert not np.any(ok & ~exact(rho, a, cap, rho_min)), "pre-test accepted a cell the FP64 test rejects"
    return ok


def test_pretest_never_accepts_what_fp64_rejects():
    rng = np.random.default_rng(20250918)
    n = 400_000
    for cap, rho_min in ((0.25, 1e-6), (1.0, 0.2), (0.3, 0.0), (0.1, 1e-30), (0.7, 3.0)):
        rho = np.exp(rng.normal(-0.5, 3.0, n))
        # a near cap rho (relative offsets down to 2^-30) and near rho - rho_min
        rel = rng.choice([-1.0, 1.0], n) * 2.0 ** -rng.uniform(10, 30, n)
        a1 = cap * rho * (1.0 + rel)
        a2 = (rho - rho_min) * (1.0 + rel)
        a3 = cap * rho * rng.uniform(0.0, 1.2, n)
        hits = 0
        for a in (a1, a2, a3):
            a = a[a > 0]
            r = rho[: a.size]
            hits += int(_check(r, a, cap, rho_min).sum())
        assert hits > n // 4  # the fast case is taken often


def test_pretest_at_the_ends_of_the_fp32_range():
    tiny, huge = 2.0 ** -126, 2.0 ** 127
    rho = np.array([tiny, tiny * 3, 1e-39, 1e-45, huge, 1e38, 3e38, 1e300, 1e-300, 1.0])
    for frac in (1e-9, 0.1, 0.2499, 0.25, 0.2501, 0.9):
        _check(rho, rho * frac, 0.25, 0.0)
        _check(rho, rho * frac, 0.25, 1e-6)
    # a outside the FP32 range never decides
    assert not pretest(np.array([1.0]), np.array([-1e-300]), F32(0.25), F32(0.0))[0]
    assert not pretest(np.array([1e300]), np.array([-1.0]), F32(0.25), F32(0.0))[0]


def test_pretest_takes_the_common_case():
    # a small removal in an ordinary cell is decided in FP32
    assert pretest(np.array([1.0]), np.array([-0.01]), F32(0.25), round_up_f32(1e-6))[0]
    # the Fig. 1 setting (cap 1, rho_min 0.2, a = 1) is left to FP64
    assert not pretest(np.array([1.0]), np.array([-1.0]), F32(1.0), round_up_f32(0.2))[0]
