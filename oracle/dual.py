"""Forward-mode derivatives of one supernova pass -- TEST INFRASTRUCTURE ONLY.

A second restatement of the supernova deposit (Sec. 3.2.1, Eq. du, v_COM,
Eq. dp, Eq. psnr) in pure Python on dual numbers (value, tangent), for small
boxes.  The kernel cells and covered fractions omega come from the C oracle:
they are piecewise constant in the particle's position and carry no
derivative.  The tangent of the updated state is the tangent of the summed
buffer, with the limiter's eta held fixed and cells where the limiter acts
passing no tangent (the adjoint's definition).  Used to check the GPU
adjoint through the identity <J dtheta, v> = <dtheta, J^T v>.

Parity of this module is pinned against the C oracle (primal values) and
against central finite differences of the C oracle (tangents).
"""
from __future__ import annotations

import math

import numpy as np


class Dual:
    __slots__ = ("v", "t")

    def __init__(self, v, t=0.0):
        self.v, self.t = float(v), float(t)

    @staticmethod
    def of(a):
        return a if isinstance(a, Dual) else Dual(a, 0.0)

    def __add__(self, o):
        o = Dual.of(o)
        return Dual(self.v + o.v, self.t + o.t)

    __radd__ = __add__

    def __sub__(self, o):
        o = Dual.of(o)
        return Dual(self.v - o.v, self.t - o.t)

    def __rsub__(self, o):
        return Dual.of(o) - self

    def __mul__(self, o):
        o = Dual.of(o)
        return Dual(self.v * o.v, self.t * o.v + self.v * o.t)

    __rmul__ = __mul__

    def __truediv__(self, o):
        o = Dual.of(o)
        return Dual(self.v / o.v, (self.t * o.v - self.v * o.t) / (o.v * o.v))

    def __rtruediv__(self, o):
        return Dual.of(o) / self

    def __neg__(self):
        return Dual(-self.v, -self.t)


def dsqrt(a):
    a = Dual.of(a)
    r = math.sqrt(a.v)
    return Dual(r, a.t / (2.0 * r) if r > 0 else 0.0)


def dpow(a, e):
    a = Dual.of(a)
    r = a.v ** e
    return Dual(r, e * a.v ** (e - 1.0) * a.t)


def pass_tangent(orc, params, box, state, parts, tangents, passmask):
    """Value and tangent of the summed buffer's contribution to the updated
    state (valid cells, arrays (5, nz, ny, nx)), along `tangents` (dict of
    per-particle tangents of m, e, px, py, pz, x, y, z).  `passmask` (nz, ny,
    nx): 1 where the limiter left the cell unscaled."""
    nx, ny, nz = box.n
    val = np.zeros((5, nz, ny, nx))
    tan = np.zeros((5, nz, ny, nx))
    U = box.valid(state)
    V = 1.0
    for s in range(len(parts["x"])):
        th = {k: Dual(parts[k][s], tangents[k][s]) for k in ("m", "e", "px", "py", "pz", "x", "y", "z")}
        ijk, om = orc.kernel_of(params, box, parts["x"][s], parts["y"][s], parts["z"][s])
        keep = om > 0
        ijk, om = ijk[keep], om[keep]
        sw = sr = 0.0
        sp = [0.0, 0.0, 0.0]
        for (i, j, k), w in zip(ijk, om):
            u = U[:, k % nz, j % ny, i % nx]
            sw += w
            sr += w * u[0]
            for a in range(3):
                sp[a] += w * u[1 + a]
        Vsnr = sw * V
        m, pe, E = th["m"], [th["px"], th["py"], th["pz"]], th["e"]
        Msnr = sr * V + m
        vc = [(sp[a] * V + pe[a]) / Msnr for a in range(3)]
        nH = Msnr / (params["mu_H"] * Vsnr)
        Msf = params["A_sf"] * dpow(nH, -0.26)
        RM = (Msnr / Msf).v
        if RM <= params["RM_ej"]:
            prad = Dual(0.0)
        elif RM <= params["RM_st"]:
            prad = dsqrt(2.0 * m * params["eps_K"] * E)
        else:
            prad = params["A_p"] * dpow(nH, -0.17)
        Ekin = (pe[0] * pe[0] + pe[1] * pe[1] + pe[2] * pe[2]) / (2.0 * m)
        q = m / Vsnr
        e = (E + Ekin) / Vsnr
        Pv = prad / Vsnr
        xs = [th["x"], th["y"], th["z"]]
        for (i, j, k), w in zip(ijk, om):
            c = (k % nz, j % ny, i % nx)
            u = U[:, c[0], c[1], c[2]]
            d = [(float(cc) + 0.5) - xx for cc, xx in zip((i, j, k), xs)]
            dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2]
            if dd.v > 0:
                dist = dsqrt(dd)
                sc = (w * Pv) / dist
            else:
                sc = Dual(0.0)
            pr = [sc * d[a] for a in range(3)]
            rn = u[0] + q
            dU = [w * q] + [w * (rn * vc[a] - u[1 + a]) + pr[a] for a in range(3)]
            dU.append(w * e + (vc[0] * pr[0] + vc[1] * pr[1] + vc[2] * pr[2]))
            for f in range(5):
                val[(f,) + c] += dU[f].v
                if passmask[c]:
                    tan[(f,) + c] += dU[f].t
    return val, tan
