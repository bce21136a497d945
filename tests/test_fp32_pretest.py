"""Soundness of the FP32 decisions of the kernels: the limiters' pre-tests
(k_sink_eta_apply and k_apply_fb_stream: whenever one decides eta = 1, the
FP64 test agrees) and the plan's kernel-membership, full-cell and sub-point
decisions (taken in FP32 outside a 2^-14 band around r_K^2, each equal to the
FP64 decision of the canonical order).

Sink pre-test (accretion limiter of Sec. 3.1.1):

The kernel decides the common case eta = 1 of the accretion limiter
(Sec. 3.1.1) in FP32: a value truncated from FP64 to FP32, cap rounded down,
rho_min rounded up, and a 2^-16 relative margin on each comparison.  It must
never say "eta = 1" where the FP64 tests a <= RN(cap rho) and
a <= RN(rho - rho_min) fail.  numpy's float32 operations are IEEE
round-to-nearest, like the GPU's FP32 pipe without contraction, so the
pre-test restated here runs the same operations; the inputs crowd the two
decision boundaries and the ends of the FP32 range.
"""
import math

import numpy as np
import pytest

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


# ---------------------------------------------------------------------------
# the supernova apply's FP32 pre-check of Eq. lambda (k_apply_fb_stream)
# ---------------------------------------------------------------------------

def sn_pretest(U, D):
    """The kernel's FP32 test that the constraint of Eq. lambda holds at
    lambda = 1: f = e_int0 rho'/rho + |p + dp|^2/(2 rho') - E' < -2^-14 M,
    on values truncated to FP32, with rho' >= rho and M in a safe range."""
    with np.errstate(all="ignore"):
        r, p0, p1, p2, E = (f32_trunc(U[i]) for i in range(5))
        dr, d0, d1, d2, dE = (f32_trunc(D[i]) for i in range(5))
        r1, E1 = r + dr, E + dE
        pp = (p0 * p0 + p1 * p1) + p2 * p2
        k0 = pp / (F32(2.0) * r)
        q = r1 / r
        n0, n1, n2 = p0 + d0, p1 + d1, p2 + d2
        kn = ((n0 * n0 + n1 * n1) + n2 * n2) / (F32(2.0) * r1)
        f = ((E - k0) * q + kn) - E1
        M = (np.abs(E) + k0) * q + kn + np.abs(E1)
        return (dr >= F32(0)) & (M > F32(1e-30)) & (M < F32(1e30)) & (f < F32(-6.103515625e-05) * M)


def sn_holds_fp64(U, D):
    """Eq. lambda's constraint at lambda = 1 in the FP64 order of the limiter."""
    rho1 = U[0] + D[0]
    E1 = U[4] + D[4]
    p2 = (U[1] * U[1] + U[2] * U[2]) + U[3] * U[3]
    eint0 = U[4] - p2 / (2.0 * U[0])
    pn = [U[1] + D[1], U[2] + D[2], U[3] + D[3]]
    pnn = (pn[0] * pn[0] + pn[1] * pn[1]) + pn[2] * pn[2]
    therm = (eint0 * rho1) / U[0]
    return therm + pnn / (2.0 * rho1) <= E1


def test_supernova_pretest_never_accepts_what_fp64_rejects():
    rng = np.random.default_rng(918261)
    n = 300_000
    rho = np.exp(rng.normal(-0.5, 2.0, n))
    p = rng.normal(0, 0.5, (3, n)) * rho
    eint = rho * np.exp(rng.normal(0.0, 2.0, n))
    E = eint + (p * p).sum(0) / (2 * rho)
    drho = rho * np.exp(rng.uniform(-12, 0, n))
    dp = rng.normal(0, 1.0, (3, n)) * rho
    U = np.stack([rho, p[0], p[1], p[2], E])
    # energy deposit that puts the cell near the constraint's boundary
    rho1 = rho + drho
    pn = p + dp
    need = eint * rho1 / rho + (pn * pn).sum(0) / (2 * rho1) - E
    rel = rng.choice([-1.0, 1.0], n) * 2.0 ** -rng.uniform(3, 40, n)
    dE = need * (1.0 + rel) + np.abs(need) * rel
    D = np.stack([drho, dp[0], dp[1], dp[2], dE])
    ok = sn_pretest(U, D)
    exact = np.array([sn_holds_fp64(U[:, i], D[:, i]) for i in np.nonzero(ok)[0]])
    assert exact.all(), "pre-check accepted a cell the FP64 test rejects"
    assert ok.sum() > n // 10  # the fast case is taken often


# ---------------------------------------------------------------------------
# the plan's FP32 membership and sub-point decisions (plan_particle)
# ---------------------------------------------------------------------------

def _band(r2):
    lo, hi = r2 * (1.0 - 2.0 ** -14), r2 * (1.0 + 2.0 ** -14)
    blo, bhi = F32(lo), F32(hi)
    if float(blo) > lo:
        blo = np.nextafter(blo, F32(0))
    if float(bhi) < hi:
        bhi = np.nextafter(bhi, F32(3e38))
    return blo, bhi


def _plan_decisions(x, rK, S):
    """For particles at x (n, 3), FP64: the kernel's FP32 decisions, restated
    with the same operations: per-axis squares of ((o - R) - f) + 1/2 and of
    ((o - R) - f) + (a + 1/2)/S, f = x - floor(x) rounded to FP32; a centre is
    in when (sx + sy) + sz < band_lo, out when > band_hi; a sub-point is
    summed as (sy + sz) + sx.  Returns the decisions with the FP64 truth for
    every (particle, offset) and (particle, offset, sub-point)."""
    R = int(math.ceil(rK))
    W = 2 * R + 1
    r2 = rK * rK
    blo, bhi = _band(r2)
    h = np.floor(x)
    f = (x - h).astype(np.float32)                        # (n, 3)
    o = (np.arange(W) - R).astype(np.float32)             # (W,)
    e = (o[None, None, :] - f[:, :, None])                 # (n, 3, W), FP32
    csq = (e + F32(0.5)) * (e + F32(0.5))
    tf = (csq[:, 0, None, None, :] + csq[:, 1, None, :, None]) + csq[:, 2, :, None, None]  # (n, z, y, x)
    # FP64 truth at the centres, in the canonical order
    oo = np.arange(W) - R
    d = (h[:, :, None] + oo[None, None, :] + 0.5) - x[:, :, None]    # (n, 3, W), FP64
    d2 = (d[:, 0, None, None, :] ** 2 + d[:, 1, None, :, None] ** 2) + d[:, 2, :, None, None] ** 2
    fr = np.array([(a + 0.5) / S for a in range(S)])
    frf = fr.astype(np.float32)
    u = e[:, :, :, None] + frf[None, None, None, :]        # (n, 3, W, S), FP32
    sub = u * u
    ds = (h[:, :, None, None] + oo[None, None, :, None] + fr[None, None, None, :]) - x[:, :, None, None]
    return (tf, blo, bhi, d2, r2, sub, ds)


@pytest.mark.parametrize("rK,S", [(2.0, 4), (4.0, 1), (2.5, 2), (3.0, 8)])
def test_plan_fp32_decisions_equal_the_fp64_ones(rK, S):
    rng = np.random.default_rng(int(rK * 10) + S)
    n = 2000
    R = int(math.ceil(rK))
    # random particles, and particles placed so that one centre sits within
    # 2^-30 .. 2^-10 (relative) of r_K
    xr = rng.uniform(0, 64, (n, 3))
    off = rng.integers(-R, R + 1, (n, 3)).astype(float)
    dirs = rng.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    rel = rng.choice([-1.0, 1.0], n) * 2.0 ** -rng.uniform(10, 30, n)
    centre = 20.5 + off
    xt = centre - dirs * (rK * (1.0 + rel))[:, None]
    x = np.concatenate([xr, xt])
    tf, blo, bhi, d2, r2, sub, ds = _plan_decisions(x, rK, S)
    inside = d2 < r2
    assert np.all(inside[tf < blo]), "FP32 'in' where FP64 says out"
    assert not np.any(inside[tf > bhi]), "FP32 'out' where FP64 says in"
    assert np.count_nonzero((tf >= blo) & (tf <= bhi)) > 0  # the band is exercised
    # sub-points: (sy + sz) + sx against the band, on a subset (memory)
    W = 2 * R + 1
    m = max(64, int(2e7 // (W ** 3 * S ** 3)))
    pick = np.concatenate([np.arange(min(m // 2, n)), n + np.arange(min(m // 2, n))])
    sb, db = sub[pick], ds[pick]
    v = (sb[:, 1][:, None, :, None, None, :, None] + sb[:, 2][:, :, None, None, :, None, None]) + \
        sb[:, 0][:, None, None, :, None, None, :]
    t64 = (db[:, 0][:, None, None, :, None, None, :] ** 2 + db[:, 1][:, None, :, None, None, :, None] ** 2) + \
        db[:, 2][:, :, None, None, :, None, None] ** 2
    sin = t64 < r2
    assert np.all(sin[v < blo]), "FP32 sub-point 'in' where FP64 says out"
    assert not np.any(sin[v > bhi]), "FP32 sub-point 'out' where FP64 says in"
    # "full" cells (omega = 1 without counting): the per-axis larger of the
    # first and last sub-point squares, summed, below band_lo
    fc = np.maximum(sb[..., 0], sb[..., S - 1])          # (m, 3, W)
    full = (fc[:, 0][:, None, None, :] + fc[:, 1][:, None, :, None]) + fc[:, 2][:, :, None, None] < blo
    every = sin.reshape(sin.shape[:4] + (-1,)).all(axis=4)
    assert np.all(every[full]), "a cell taken as full has a sub-point outside"
    assert full.any()
