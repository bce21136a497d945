"""Pins of the oracle's sink creation (Sec. 3.1.2) to facts from outside it:

- brute force over a periodic box (numpy rolls): the created cells are
  exactly the strict local density maxima within r_K whose retained
  accretion buffer is zero and whose density exceeds rho_Tr (uniform here up
  to rounding, because the gas has one specific thermal energy);
- conservation: the mass and momentum a created sink carries are the ones
  its cell lost (Eq. conservation);
- the cell keeps its velocity and specific energy, and the sink moves with
  the cell (Sec. 3.1.2);
- two peaks closer than r_K make one sink (the higher), two peaks farther
  apart make two, two equal peaks closer than r_K make none (neither is a
  strict maximum), and a peak inside an accretion kernel makes none.
"""
import math

import numpy as np
import pytest

from paper_2509_18261_gb300 import synthetic as syn


def _offsets(rK):
    R = int(math.ceil(rK))
    return [(ox, oy, oz) for oz in range(-R, R + 1) for oy in range(-R, R + 1) for ox in range(-R, R + 1)
            if (ox, oy, oz) != (0, 0, 0) and ox * ox + oy * oy + oz * oz < rK * rK]


def _brute_local_max(rho, rK):
    """rho[z, y, x] on a periodic box: strict maximum over the r_K sphere."""
    ok = np.ones(rho.shape, dtype=bool)
    for ox, oy, oz in _offsets(rK):
        ok &= rho > np.roll(rho, shift=(-oz, -oy, -ox), axis=(0, 1, 2))
    return ok


def _state(seed, n, peaks=()):
    rng = np.random.default_rng(seed)
    box = syn.Box((n, n, n), 4)
    st = syn.gas_state(rng, box)
    v = box.valid(st)
    for (i, j, k), f in peaks:
        v[:, k, j, i] *= f  # scaling all fields keeps velocity and specific energy
    return box, st


def test_created_cells_match_brute_force(orc):
    box, st = _state(3, 14)
    params = syn.sink_params(G=0.3)
    buf = box.empty(0.0)
    bv = box.valid(buf)
    rng = np.random.default_rng(9)
    bv[:, rng.random(bv.shape[1:]) < 0.3] = 1e-3  # some cells lie in accretion kernels
    rho0 = box.valid(st)[0].copy()
    st2 = st.copy()
    n, new = orc.create_sinks(params, box, st2, buf)
    assert n > 3
    cells = [(int(z), int(y), int(x)) for x, y, z in zip(new["x"], new["y"], new["z"])]
    # one specific thermal energy: one rho_Tr, up to the rounding of
    # e_int / rho (a few ulp)
    rho_tr = np.array([float(box.valid(st2)[0][c]) for c in cells])
    thr = float(np.median(rho_tr))
    assert np.all(np.abs(rho_tr - thr) <= 1e-14 * thr)
    assert not np.any(np.abs(rho0 - thr) <= 1e-12 * thr)  # no cell at the threshold
    want = _brute_local_max(rho0, params["r_K"]) & np.all(bv == 0, axis=0) & (rho0 > thr)
    got = np.zeros_like(want)
    for c in cells:
        got[c] = True
    assert np.array_equal(got, want)
    # sink positions are cell centres, in cell index order
    keys = [c[0] * 10000 + c[1] * 100 + c[2] for c in cells]
    assert keys == sorted(keys)
    assert np.all(new["x"] % 1.0 == 0.5)


@pytest.mark.parametrize("dx", [1.0, 0.5])
def test_conservation_and_cell_velocity(orc, dx):
    box, st = _state(5, 12)
    params = syn.sink_params(G=0.3 / dx ** 2)  # the same rho_Tr at either cell size
    buf = box.empty(0.0)
    before = box.valid(st).copy()
    st2 = st.copy()
    n, new = orc.create_sinks(params, box, st2, buf, dx=dx)
    assert n > 0
    after = box.valid(st2)
    V = dx ** 3
    for f, key in ((0, "m"), (1, "px"), (2, "py"), (3, "pz")):
        lost = math.fsum(float(v) for v in (before[f] - after[f]).ravel()) * V
        gained = math.fsum(float(v) for v in new[key])
        scale = math.fsum(abs(float(v)) for v in new[key]) + 1e-300
        assert abs(lost - gained) <= 1e-14 * scale + 1e-15 * abs(lost), key
    changed = np.any(after != before, axis=0)
    assert changed.sum() == n
    for f in (1, 2, 3, 4):
        a = after[f][changed] / after[0][changed]
        b = before[f][changed] / before[0][changed]
        assert np.allclose(a, b, rtol=4e-16, atol=0)
    for a, key in enumerate(("px", "py", "pz")):
        k = np.argwhere(changed)
        vcell = np.array([before[1 + a][tuple(c)] / before[0][tuple(c)] for c in k])
        assert np.allclose(new[key] / new["m"], vcell, rtol=4e-16, atol=0)


def _uniform(n, peaks):
    """Gas at rest with rho = 1, E = 1 and the listed cells scaled."""
    box = syn.Box((n, n, n), 4)
    st = box.empty(np.nan)
    v = box.valid(st)
    v[0], v[1], v[2], v[3], v[4] = 1.0, 0.0, 0.0, 0.0, 1.0
    for (i, j, k), f in peaks:
        v[:, k, j, i] *= f
    return box, st


def test_peaks_and_kernels():
    import oracle

    params = syn.sink_params(G=0.3)
    n = 16
    _state = lambda seed, n, peaks: _uniform(n, peaks)  # noqa: E731
    # two peaks 3 cells apart (< r_K = 4): the higher one only
    box, st = _state(1, n, peaks=[((4, 4, 4), 40.0), ((7, 4, 4), 50.0)])
    cnt, new = oracle.create_sinks(params, box, st.copy(), box.empty(0.0))
    cells = set(zip(new["x"] - 0.5, new["y"] - 0.5, new["z"] - 0.5))
    assert (7.0, 4.0, 4.0) in cells and (4.0, 4.0, 4.0) not in cells
    # two peaks 8 cells apart: both
    box, st = _state(1, n, peaks=[((4, 4, 4), 40.0), ((12, 4, 4), 50.0)])
    cnt, new = oracle.create_sinks(params, box, st.copy(), box.empty(0.0))
    cells = set(zip(new["x"] - 0.5, new["y"] - 0.5, new["z"] - 0.5))
    assert {(4.0, 4.0, 4.0), (12.0, 4.0, 4.0)} <= cells
    # the same peak inside an accretion kernel (non-zero summed buffer): none
    buf = box.empty(0.0)
    box.valid(buf)[0, 4, 4, 4] = -1e-9
    cnt, new = oracle.create_sinks(params, box, st.copy(), buf)
    cells = set(zip(new["x"] - 0.5, new["y"] - 0.5, new["z"] - 0.5))
    assert (4.0, 4.0, 4.0) not in cells and (12.0, 4.0, 4.0) in cells
    # two equal peaks 2 cells apart: neither is a strict local maximum, none
    box, st = _state(1, n, peaks=[((4, 4, 4), 40.0), ((6, 4, 4), 40.0), ((12, 4, 4), 50.0)])
    rho = box.valid(st)[0]
    assert not _brute_local_max(rho, params["r_K"])[4, 4, 4]
    cnt, new = oracle.create_sinks(params, box, st.copy(), box.empty(0.0))
    cells = set(zip(new["x"] - 0.5, new["y"] - 0.5, new["z"] - 0.5))
    assert (4.0, 4.0, 4.0) not in cells and (6.0, 4.0, 4.0) not in cells and (12.0, 4.0, 4.0) in cells
    # two peaks exactly r_K = 4 cells apart: neither lies within r_K of the
    # other (the strict "< r_K" of kernel membership), so both
    box, st = _state(1, n, peaks=[((4, 4, 4), 40.0), ((8, 4, 4), 50.0)])
    cnt, new = oracle.create_sinks(params, box, st.copy(), box.empty(0.0))
    cells = set(zip(new["x"] - 0.5, new["y"] - 0.5, new["z"] - 0.5))
    assert {(4.0, 4.0, 4.0), (8.0, 4.0, 4.0)} <= cells
    # peaks at the two faces of the x axis, one cell apart through the face:
    # on a periodic axis the higher one only; on a non-periodic axis nothing
    # lies beyond the face, both are maxima
    box, st = _state(1, n, peaks=[((0, 4, 4), 40.0), ((15, 4, 4), 50.0)])
    cnt, new = oracle.create_sinks(params, box, st.copy(), box.empty(0.0))
    cells = set(zip(new["x"] - 0.5, new["y"] - 0.5, new["z"] - 0.5))
    assert (15.0, 4.0, 4.0) in cells and (0.0, 4.0, 4.0) not in cells
    cnt, new = oracle.create_sinks(params, box, st.copy(), box.empty(0.0), periodic=(0, 1, 1))
    cells = set(zip(new["x"] - 0.5, new["y"] - 0.5, new["z"] - 0.5))
    assert {(0.0, 4.0, 4.0), (15.0, 4.0, 4.0)} <= cells
