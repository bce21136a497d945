"""Error bounds that set the tolerances of the atomic-mode parity tests.

The atomic deposit adds the same terms as the oracle in another order, so a
summed buffer value differs from the oracle's by at most tau * A_c per cell
and field, A_c = sum_s |Delta U^s_c| (tau = 1e-12, the buffer tolerance; the
reordering itself gives at most about 2 (k - 1) u A_c for k contributions,
u = 2^-53).  What that buffer difference does to the state after Step 5, to
the limiter's eta and to the sinks after Step 4 is bounded here by a running
(first-order) error analysis of the same formulas in the same operation
order as the kernels and the oracle: every value carries a bound on its
distance from the exact result of exact inputs, propagated through each
operation by its partial derivatives, plus u |result| for the operation's own
rounding.  Where a decision of the limiter (the root test of Eq. lambda, its
discriminant, the bracket [0, 1]) lies within the bound of its operands, the
cell is flagged ambiguous: there the limiter itself is discontinuous and
either side's result is a correct evaluation.

Test infrastructure only: the library never imports this module.
"""
from __future__ import annotations

import numpy as np

U_ROUND = 2.0 ** -53  # unit roundoff of FP64
SAFETY = 2.0          # first-order bounds are doubled to cover second-order terms


class RV:
    """A value (FP64 array, evaluated as the kernels evaluate it) with a bound
    on its distance from the exact result."""

    __slots__ = ("v", "e")

    def __init__(self, v, e=None):
        self.v = np.asarray(v, dtype=np.float64)
        self.e = np.zeros_like(self.v) if e is None else np.asarray(e, dtype=np.float64)

    def __add__(self, o):
        o = _rv(o)
        z = self.v + o.v
        return RV(z, self.e + o.e + U_ROUND * np.abs(z))

    def __sub__(self, o):
        o = _rv(o)
        z = self.v - o.v
        return RV(z, self.e + o.e + U_ROUND * np.abs(z))

    def __mul__(self, o):
        o = _rv(o)
        z = self.v * o.v
        return RV(z, np.abs(o.v) * self.e + np.abs(self.v) * o.e + self.e * o.e + U_ROUND * np.abs(z))

    def __truediv__(self, o):
        o = _rv(o)
        with np.errstate(divide="ignore", invalid="ignore"):
            z = self.v / o.v
            den = np.abs(o.v) - o.e
            e = np.where(den > 0, (self.e + np.abs(z) * o.e) / np.where(den > 0, den, 1.0), np.inf)
        return RV(z, e + U_ROUND * np.abs(z))

    def __neg__(self):
        return RV(-self.v, self.e)


def _rv(x):
    return x if isinstance(x, RV) else RV(x)


def rsqrt_free_sqrt(x):
    """sqrt with |sqrt(x + d) - sqrt(x)| <= min(|d| / (2 sqrt(x)), sqrt(|d|))."""
    with np.errstate(invalid="ignore", divide="ignore"):
        z = np.sqrt(np.maximum(x.v, 0.0))
        lin = np.where(z > 0, x.e / (2.0 * np.where(z > 0, z, 1.0)), np.inf)
        e = np.minimum(lin, np.sqrt(x.e))
    return RV(z, e + U_ROUND * z)


def sn_lambda_bound(U, D, dD):
    """lambda of Eq. lambda for cells U, D (arrays (5, n)) evaluated as the
    kernels do, with a bound on |lambda - lambda*(D*)| for every exact buffer
    D* within dD (5, n) of D.  Returns (lam, bound, ambiguous, noroot)."""
    U = [RV(U[f]) for f in range(5)]
    Dv = [RV(D[f], dD[f]) for f in range(5)]
    n = U[0].v.shape
    lam = np.ones(n)
    bound = np.zeros(n)
    amb = np.zeros(n, dtype=bool)
    noroot = np.zeros(n, dtype=bool)
    zero_dp = (D[1] == 0.0) & (D[2] == 0.0) & (D[3] == 0.0)
    rho1 = U[0] + Dv[0]
    E1 = U[4] + Dv[4]
    p2 = (U[1] * U[1] + U[2] * U[2]) + U[3] * U[3]
    eint0 = U[4] - p2 / (RV(2.0) * U[0])
    pn = [U[1 + a] + Dv[1 + a] for a in range(3)]
    pn2 = (pn[0] * pn[0] + pn[1] * pn[1]) + pn[2] * pn[2]
    therm = (eint0 * rho1) / U[0]
    lhs = therm + pn2 / (RV(2.0) * rho1)
    gap = lhs - E1
    at_one = gap.v <= 0.0                     # constraint holds at lambda = 1
    unsure_one = np.abs(gap.v) <= gap.e       # ... or might, within the bound
    A = (Dv[1] * Dv[1] + Dv[2] * Dv[2]) + Dv[3] * Dv[3]
    B = (U[1] * Dv[1] + U[2] * Dv[2]) + U[3] * Dv[3]
    C = p2 - (RV(2.0) * rho1) * (E1 - therm)
    disc = B * B - A * C
    sq = rsqrt_free_sqrt(disc)
    Bpos = B.v >= 0.0
    Qp = -(B + sq)
    Qn = sq - B
    hi_p = C / Qp
    lo_p = Qp / A
    hi_n = Qn / A
    lo_n = C / Qn
    # the two forms of the quadratic formula agree in exact arithmetic: where
    # the sign of B is unsure, either side may take either form
    Bunsure = np.abs(B.v) <= B.e
    hi = RV(np.where(Bpos, np.where(Qp.v != 0.0, hi_p.v, 0.0), hi_n.v),
            np.where(Bunsure, np.maximum(hi_p.e, hi_n.e), np.where(Bpos, hi_p.e, hi_n.e)))
    lo = RV(np.where(Bpos, lo_p.v, lo_n.v),
            np.where(Bunsure, np.maximum(lo_p.e, lo_n.e), np.where(Bpos, lo_p.e, lo_n.e)))
    with np.errstate(invalid="ignore"):
        nr_disc = ~(disc.v >= 0.0)
        nr_br = (hi.v < 0.0) | (lo.v > 1.0)
        unsure_root = (np.abs(disc.v) <= disc.e) | (np.abs(hi.v) <= hi.e) | (np.abs(lo.v - 1.0) <= lo.e) | \
            ~np.isfinite(hi.e)
    root = np.minimum(hi.v, 1.0)
    root_e = hi.e
    lam_root = np.where(nr_disc | nr_br, 0.0, root)
    lim = ~zero_dp & ~at_one
    lam = np.where(lim, lam_root, 1.0)
    noroot = lim & (nr_disc | nr_br)
    bound = np.where(lim & ~(nr_disc | nr_br), root_e, 0.0)
    # lambda = 1 on one side, the root on the other: the root is within its
    # bound of 1 there (the quadratic vanishes at lambda = 1 when lhs = E1)
    near = ~zero_dp & unsure_one
    with np.errstate(invalid="ignore"):
        bound = np.where(near, np.maximum(bound, np.abs(1.0 - np.where(nr_disc | nr_br, 0.0, root)) + root_e), bound)
    amb = ~zero_dp & (~at_one | unsure_one) & (unsure_root | ~np.isfinite(bound))
    bound = np.where(amb, 1.0, np.minimum(SAFETY * bound, 1.0))
    return lam, bound, amb, noroot


def feedback_state_tolerance(U, D, A, tau=1e-12, dD=None):
    """Per cell and field, the largest |U_new(GPU) - U_new(oracle)| after
    Step 5 of a supernova pass when both buffers lie within tau * A of the
    exact sum (or within dD, when given).  U, D, A: arrays (5, n) of the
    pre-update state, the oracle's summed buffer and the oracle's sum of
    |Delta U|.  Returns (tol, ambiguous)."""
    dD = tau * A if dD is None else dD
    lam, bl, amb, _ = sn_lambda_bound(U, D, dD)
    unew = np.abs(U) + np.abs(D)
    tol = dD + 2.0 * U_ROUND * unew + 2.0 * U_ROUND * np.abs(D)
    for f in (1, 2, 3):
        # U + lambda D on both sides: |D| |d lambda| + lambda |dD|
        tol[f] = 2.0 * bl * (np.abs(D[f]) + dD[f]) + lam * dD[f] + 2.0 * U_ROUND * (unew[f] + np.abs(D[f]))
    return tol, amb


def sink_state_tolerance(U, D, A, eta, tau=1e-12, dD=None, dlim=None):
    """As feedback_state_tolerance for a sink pass.  eta (n,) is the oracle's.
    Where the limiter acts, eta = a_lim / a with a_lim a function of the
    state alone and a = -D_rho, whose relative error is tau (every term of
    D_rho is negative, so A_rho = a): eta moves by at most eta (tau + 2u)
    (plus dlim / a when a_lim is itself known only to within dlim)."""
    dD = tau * A if dD is None else dD
    deta = eta * (np.max(dD[0:1] / np.maximum(A[0:1], 1e-300), axis=0) + 4.0 * U_ROUND)
    if dlim is not None:
        # a_lim itself known only to within dlim (two evaluations of rho_Tr)
        deta = deta + dlim / np.maximum(np.abs(D[0]), 1e-300)
    unew = np.abs(U) + np.abs(D)
    tol = eta * dD + np.abs(D) * deta + 4.0 * U_ROUND * (unew + np.abs(D))
    return tol


def sink_return_tolerance(m0, m_new, p_new, vmax, ncells, tau=1e-12):
    """Bound on |u_s(GPU) - u_s(oracle)| after Step 4 for one sink: both sides
    add the same removals b = eta a V in the same kernel order and differ
    only through eta (relative tau + 2u per cell, as above) and the rounding
    of those sums (ncells terms).  The removed mass sum_c b is |m_new - m0|;
    momentum terms are b v with |v| <= vmax over the sink's kernel cells."""
    rel = tau + 4.0 * U_ROUND + 2.0 * ncells * U_ROUND
    dm = np.abs(m_new - m0)
    tm = rel * dm + 4.0 * U_ROUND * np.abs(m_new)
    tp = rel * dm * vmax + 4.0 * U_ROUND * np.abs(p_new)
    return tm, tp
