"""Pins of the oracle's particle-mesh (PM/PIC) deposit, the Step subset of
Sec. 2.2 that uses Steps 1, 2 and 5 only, to facts from outside the oracle:

- conservation: every particle's (m, p, e) arrives on the mesh
  (Eq. conservation), checked with an exactly rounded sum;
- the split over a particle's kernel cells is proportional to the covered
  fraction omega, counted here by brute force over the sub-points;
- no limiter: U_new = U_old + Delta U^sum cell by cell, and the particles are
  not changed (Sec. 2.2: "interactions do not modify particle properties").
"""
import math

import numpy as np
import pytest

from paper_2509_18261_gb300 import synthetic as syn


def _case(seed=4, n=12, count=300):
    rng = np.random.default_rng(seed)
    box = syn.Box((n, n, n), 4)
    state = syn.gas_state(rng, box)
    parts = syn.particles(rng, box.n, count, "feedback", clustered=150, nclusters=3)
    return box, state, parts


@pytest.mark.parametrize("dx", [1.0, 0.5])
def test_mass_momentum_energy_arrive_on_the_mesh(orc, dx):
    """Sum over cells of Delta U times V = dx^3 returns each particle's (m, p,
    e), for any cell size."""
    box, state, parts = _case()
    params = syn.mass_params()
    st = state.copy()
    r = orc.cycle(params, box, st, {k: v.copy() for k, v in parts.items()}, dx=dx)
    V = dx ** 3
    dU = box.valid(st) - box.valid(state)
    for f, key in enumerate(("m", "px", "py", "pz", "e")):
        got = math.fsum(float(v) for v in dU[f].ravel()) * V
        want = math.fsum(float(v) for v in parts[key])
        A = math.fsum(abs(float(v)) for v in parts[key])
        assert abs(got - want) <= 1e-13 * A, key
    assert r["counts"][0] == 0  # nothing limited


def _brute_omega(x, y, z, i, j, k, rK, S):
    cnt = 0
    for c in range(S):
        for b in range(S):
            for a in range(S):
                sx = (i + (a + 0.5) / S) - x
                sy = (j + (b + 0.5) / S) - y
                sz = (k + (c + 0.5) / S) - z
                if (sx * sx + sy * sy) + sz * sz < rK * rK:
                    cnt += 1
    return cnt / S ** 3


def test_split_follows_the_covered_fraction(orc):
    box = syn.Box((10, 10, 10), 4)
    state = syn.gas_state(np.random.default_rng(2), box)
    one = {k: np.array([v]) for k, v in dict(x=4.3, y=5.7, z=5.05, m=2.0, px=0.3, py=-0.1, pz=0.2, e=1.5).items()}
    params = syn.mass_params()
    ijk, dU = orc.deltas(params, box, state, one)
    om = np.array([_brute_omega(4.3, 5.7, 5.05, i, j, k, params["r_K"], params["subsample"]) for i, j, k in ijk])
    assert np.all(om > 0)
    VK = om.sum()  # V = 1
    for f, key in enumerate(("m", "px", "py", "pz", "e")):
        want = om * (one[key][0] / VK)
        assert np.allclose(dU[:, f], want, rtol=4e-16 * 8, atol=0), key


def test_no_limiter_and_particles_unchanged(orc):
    box, state, parts = _case(seed=9)
    params = syn.mass_params()
    p = {k: v.copy() for k, v in parts.items()}
    st = state.copy()
    r = orc.cycle(params, box, st, p)
    want = box.valid(state) + box.valid(r["buf"])
    touched = np.any(box.valid(r["buf"]) != 0, axis=0)
    assert np.array_equal(box.valid(st)[:, touched], want[:, touched])
    assert np.array_equal(box.valid(st)[:, ~touched], box.valid(state)[:, ~touched])
    for k in parts:
        assert np.array_equal(p[k], parts[k])
