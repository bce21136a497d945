"""The error bounds behind the atomic-mode tolerances (tests/bounds.py),
checked on the CPU against what they claim:

- lambda of Eq. lambda evaluated in FP64 lies within its bound of the exact
  root (50-digit arithmetic) of the exact quadratic;
- two FP64 evaluations on buffers that differ by up to tau * A_c differ by
  at most the sum of their bounds;
- the same holds at cells built to sit on the limiter's decision boundaries:
  the constraint tight at lambda = 1, a double root of the quadratic, and a
  root at 0;
- the bound is not vacuous on the supernova workload: over its
  limiter-active cells it stays far below 1 except at flagged cells.
"""
import mpmath
import numpy as np
import pytest

from bounds import U_ROUND, feedback_state_tolerance, sn_lambda_bound

from paper_2509_18261_gb300 import synthetic as syn

mpmath.mp.dps = 50


def _exact_lambda(U, D):
    """Largest root in [0, 1] of the quadratic of Eq. lambda in 50-digit
    arithmetic (lambda = 1 if the constraint holds there, 0 if no root)."""
    m = mpmath.mpf
    U = [m(float(v)) for v in U]
    D = [m(float(v)) for v in D]
    if D[1] == 0 and D[2] == 0 and D[3] == 0:
        return 1.0
    rho1 = U[0] + D[0]
    E1 = U[4] + D[4]
    p2 = U[1] ** 2 + U[2] ** 2 + U[3] ** 2
    eint0 = U[4] - p2 / (2 * U[0])
    pn2 = sum((U[1 + a] + D[1 + a]) ** 2 for a in range(3))
    therm = eint0 * rho1 / U[0]
    if therm + pn2 / (2 * rho1) <= E1:
        return 1.0
    A = D[1] ** 2 + D[2] ** 2 + D[3] ** 2
    B = U[1] * D[1] + U[2] * D[2] + U[3] * D[3]
    C = p2 - 2 * rho1 * (E1 - therm)
    disc = B * B - A * C
    if disc < 0:
        return 0.0
    hi = (-B + mpmath.sqrt(disc)) / A
    lo = (-B - mpmath.sqrt(disc)) / A
    if hi < 0 or lo > 1:
        return 0.0
    return float(min(hi, m(1)))


def _limited_cells(rng, n):
    """Random cells whose momentum deposit breaks the constraint at lambda = 1."""
    rho = np.exp(rng.normal(-0.5, 1.0, n))
    p = rng.normal(0, 0.1, (3, n))
    E = (p * p).sum(0) / (2 * rho) + rho * rng.uniform(0.5, 1.5, n)
    U = np.vstack([rho, p, E])
    D = np.vstack([rng.uniform(0, 0.05, n) * rho, rng.normal(0, 1.0, (3, n)) * rho,
                   rng.uniform(0.0, 0.5, n) * rho])
    A = np.abs(D) * rng.uniform(1.0, 30.0, (5, n))  # sums of |dU| over several contributions
    return U, D, A


def _check_exact(U, D, dD):
    lam, b, amb, _ = sn_lambda_bound(U, D, dD)
    for c in range(U.shape[1]):
        if amb[c]:
            continue
        ex = _exact_lambda(U[:, c], D[:, c])
        assert abs(lam[c] - ex) <= b[c], (c, lam[c], ex, b[c])
    return lam, b, amb


def _check_perturbed(rng, U, D, A, tau, reps=4):
    dD = tau * A
    lam, b, amb, _ = sn_lambda_bound(U, D, dD)
    for _ in range(reps):
        D2 = D + dD * rng.uniform(-1.0, 1.0, D.shape)
        lam2, b2, amb2, _ = sn_lambda_bound(U, D2, dD)
        ok = amb | amb2 | (np.abs(lam - lam2) <= b + b2)
        assert np.all(ok), np.argwhere(~ok)[:5]


def test_lambda_within_its_bound_of_the_exact_root():
    rng = np.random.default_rng(1)
    U, D, A = _limited_cells(rng, 400)
    lam, b, amb = _check_exact(U, D, np.zeros_like(D))
    assert np.count_nonzero(lam < 1.0) > 300
    assert np.count_nonzero(amb) <= 4
    assert np.median(b[lam < 1.0]) < 1e-14


def test_lambda_bound_covers_reordered_buffers():
    rng = np.random.default_rng(2)
    U, D, A = _limited_cells(rng, 2000)
    _check_perturbed(rng, U, D, A, 1e-12)
    _check_perturbed(rng, U, D, A, 1e-9)


def _tight_at_one(rng, n, rel):
    """Cells where the constraint holds at lambda = 1 to within rel."""
    U, D, _ = _limited_cells(rng, n)
    rho1 = U[0] + D[0]
    p2 = (U[1:4] ** 2).sum(0)
    eint0 = U[4] - p2 / (2 * U[0])
    pn2 = ((U[1:4] + D[1:4]) ** 2).sum(0)
    lhs = eint0 * rho1 / U[0] + pn2 / (2 * rho1)
    D[4] = lhs * (1.0 + rel * rng.uniform(-1, 1, n)) - U[4]
    return U, D


def _double_root(rng, n, rel):
    """Cells where B^2 - A C vanishes to within rel (the energy deposit set so
    that C = B^2 / A)."""
    U, D, _ = _limited_cells(rng, n)
    rho1 = U[0] + D[0]
    p2 = (U[1:4] ** 2).sum(0)
    eint0 = U[4] - p2 / (2 * U[0])
    therm = eint0 * rho1 / U[0]
    A = (D[1:4] ** 2).sum(0)
    B = (U[1:4] * D[1:4]).sum(0)
    C = (B * B / A) * (1.0 + rel * rng.uniform(-1, 1, n))
    # C = p2 - 2 rho1 (E1 - therm)  =>  E1 = therm + (p2 - C) / (2 rho1)
    D[4] = therm + (p2 - C) / (2 * rho1) - U[4]
    return U, D


@pytest.mark.parametrize("make", ["tight_at_one", "double_root"])
@pytest.mark.parametrize("rel", [1e-6, 1e-12, 1e-15])
def test_lambda_bound_at_the_decision_boundaries(make, rel):
    rng = np.random.default_rng(3 + int(-np.log10(rel)))
    U, D = (_tight_at_one if make == "tight_at_one" else _double_root)(rng, 300, rel)
    A = np.abs(D) * 3.0
    _check_exact(U, D, np.zeros_like(D))
    _check_perturbed(rng, U, D, A, 1e-12)


def test_bound_is_tight_on_the_supernova_workload(orc):
    """On the 64^3 shrink of the 512^3 workload (particle density kept), the
    bound of the state after Step 5 at limiter-active cells is a small
    multiple of tau * A_c, not a blanket band."""
    w = syn.make_workload("c5_512", n=64, count_scale=(64 / 512) ** 3)
    box, params, parts = w["box"], w["fb_params"], w["fb"]
    st = w["state"].copy()
    r = orc.cycle(params, box, st, {k: v.copy() for k, v in parts.items()}, want_abs=True, want_eta=True)
    U = box.valid(w["state"]).reshape(5, -1)
    D = box.valid(r["buf"]).reshape(5, -1)
    A = box.valid(r["absbuf"]).reshape(5, -1)
    lim = r["eta"] < 1.0
    assert lim.sum() > 100
    tol, amb = feedback_state_tolerance(U[:, lim], D[:, lim], A[:, lim])
    assert np.count_nonzero(amb) == 0
    ratio = tol[1:4] / (1e-12 * A[1:4, lim] + 4 * U_ROUND * (np.abs(U[1:4, lim]) + np.abs(D[1:4, lim])))
    assert np.median(ratio) < 10.0
    assert np.all(np.isfinite(tol))
