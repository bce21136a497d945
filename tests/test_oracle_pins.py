"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each test names the passage of He et al. (2025) it checks, or the
mathematical fact (closed form, symmetry, brute force) it relies on.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2509_18261_gb300 import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def one(x, y, z, m, p=(0.0, 0.0, 0.0), e=1.0):
    d = dict(x=x, y=y, z=z, m=m, px=p[0], py=p[1], pz=p[2], e=e)
    return {k: np.array([v], dtype=np.float64) for k, v in d.items()}


def many(rows):
    keys = ("x", "y", "z", "m", "px", "py", "pz", "e")
    return {k: np.array([r[i] for r in rows], dtype=np.float64) for i, k in enumerate(keys)}


def ulp(x):
    return math.ulp(x) if x != 0 else 5e-324


def brute_members(box, x, y, z, rK):
    """All (unwrapped) buffer coordinates whose cell centre is strictly inside
    r_K of (x, y, z), found by scanning the whole padded box: no stencil
    enumerator, no wrap, no host cell."""
    g = box.g
    out = set()
    r2 = rK * rK
    for k in range(-g, box.n[2] + g):
        dz = (k + 0.5) - z
        for j in range(-g, box.n[1] + g):
            dy = (j + 0.5) - y
            for i in range(-g, box.n[0] + g):
                dx = (i + 0.5) - x
                if (dx * dx + dy * dy) + dz * dz < r2:
                    out.add((i, j, k))
    return out


# --------------------------------------------------------------------------
# elementary functions
# --------------------------------------------------------------------------

def test_exp_matches_libm_within_one_ulp(orc):
    """Cody-Waite reduction plus the degree-13 series: within 1 ulp of libm,
    including arguments whose reduced part r sits at the edge |r| = ln2/2,
    where a series one term short is off by more."""
    rng = np.random.default_rng(11)
    k = rng.integers(-1000, 1000, 4000)
    edge = k * math.log(2.0) + rng.choice([-1.0, 1.0], 4000) * rng.uniform(0.30, 0.3465, 4000)
    xs = np.concatenate([
        rng.uniform(-700.0, 700.0, 4000), rng.uniform(-1.0, 1.0, 4000), rng.uniform(-1e-9, 1e-9, 200),
        edge[np.abs(edge) < 700.0],
        [0.0, 1.0, -1.0, math.log(2.0), -math.log(2.0), 0.5 * math.log(2.0), 709.7, -707.0, -30.0, 30.0],
    ])
    worst = 0.0
    for x in xs:
        a, b = orc.exp(float(x)), math.exp(float(x))
        worst = max(worst, abs(a - b) / ulp(b))
    assert worst <= 1.0, worst
    assert orc.exp(0.0) == 1.0
    assert orc.exp(1000.0) == math.inf and orc.exp(-1000.0) == 0.0


def test_log_matches_libm_within_one_ulp(orc):
    rng = np.random.default_rng(12)
    xs = np.concatenate([
        10.0 ** rng.uniform(-300.0, 300.0, 4000), rng.uniform(0.5, 2.0, 4000), 1.0 + rng.uniform(-1e-6, 1e-6, 200),
        [1.0, 2.0, 0.5, math.e, 10.0, 1.4142135623730951, 1.4142135623730954, 5e-324, 1e-310],
    ])
    worst = 0.0
    for x in xs:
        a, b = orc.log(float(x)), math.log(float(x))
        worst = max(worst, abs(a - b) / ulp(b))
    assert worst <= 1.0, worst
    assert orc.log(1.0) == 0.0


# --------------------------------------------------------------------------
# Fig. 1 worked example (Sec. 2.2)
# --------------------------------------------------------------------------

def test_fig1_worked_example(orc):
    """Fig. 1 of Sec. 2.2: rho = 1; each sink changes each of its cells by
    -0.5; the summed buffer is -1 where the kernels overlap; the limiter
    scales it to -0.8; sinks gain the limited mass.  The per-sink -0.5 comes
    from the Truelove branch (rho - rho_Tr = 1 - 0.5) with a negligible Bondi
    rate; the floor rho_min = 0.2 with no 25% cap gives the -0.8.  The sinks
    sit on either side of the periodic x face, so Step 2 (ghost sum) joins
    their contributions as in the figure's two-block layout."""
    gold = json.load(open(os.path.join(GOLDEN, "fig1_pmp.json")))
    J = 0.25
    params = syn.sink_params(r_K=2.0, gamma=2.0, J=J, G=(J * J) * math.pi, dt=1.0, cap=1.0, rho_min=0.2)
    box = syn.Box((12, 8, 8), 2)
    rho0 = gold["rho_initial"]
    state = syn.uniform_gas(box, rho0, e_th=0.25)  # c_s^2 = 2 * 0.25 = 0.5 -> rho_Tr = 0.5
    sinks = many([(11.3, 4.5, 4.5, 1e-9, 0, 0, 0, 0), (0.9, 4.6, 4.4, 1e-9, 0, 0, 0, 0)])
    m0 = sinks["m"].copy()
    old = state.copy()
    r = orc.cycle(params, box, state, sinks, want_eta=True)

    mem = [brute_members(box, sinks["x"][s], sinks["y"][s], sinks["z"][s], 2.0) for s in range(2)]
    own = [{(i % 12, j % 8, k % 8) for (i, j, k) in m} for m in mem]
    shared = own[0] & own[1]
    assert shared, "the two kernels must overlap"
    pre = box.grid(r["pre_fold"])
    g = box.g
    for s in range(2):
        for (i, j, k) in mem[s]:
            if (i, j, k) in mem[1 - s]:
                continue
            if (i % 12, j % 8, k % 8) in own[1 - s]:
                continue  # reaches the other sink's cell through an image; summed in Step 2
            assert pre[0, k + g, j + g, i + g] == gold["delta_rho_per_sink"]
    summed = box.valid(r["buf"])
    new = box.valid(state)
    eta = r["eta"].reshape(8, 8, 12)
    for (i, j, k) in shared:
        assert summed[0, k, j, i] == gold["delta_rho_summed_overlap"]
        assert eta[k, j, i] == pytest.approx(0.8, rel=1e-15)
        assert new[0, k, j, i] - rho0 == pytest.approx(gold["delta_rho_limited_overlap"], rel=1e-14)
    for s in range(2):
        for (i, j, k) in own[s] - shared:
            assert new[0, k, j, i] == pytest.approx(rho0 + gold["delta_rho_per_sink"], rel=1e-15)
    # Step 4: each sink gains 0.5 V from its own cells and 0.8 * 0.5 V from shared ones
    for s in range(2):
        expect = 0.5 * len(own[s] - shared) + 0.4 * len(shared)
        assert sinks["m"][s] - m0[s] == pytest.approx(expect, rel=1e-14)
    # Eq. conservation: gas mass lost = sink mass gained
    dgas = math.fsum((box.valid(state)[0] - box.valid(old)[0]).ravel())
    assert dgas + math.fsum(sinks["m"] - m0) == pytest.approx(0.0, abs=1e-13 * abs(dgas))


# --------------------------------------------------------------------------
# Bondi / Bondi-Hoyle closed forms (Eq. rbh, Eq. mdot)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("Gm,r_acc,dx", [(0.1, 0.25, 1.0), (3.0, 2.0, 1.0), (1.2, 1.2, 1.0), (0.6, 1.2, 0.5)])
def test_accretion_kernel_shape(orc, Gm, r_acc, dx):
    """Gas at rest, one sink at rest, Bondi branch only: the removal per cell
    follows the Gaussian of Eq. kernel, exp(-|x_c - x_s|^2 / r_acc^2), with
    r_acc = r_BH = G m / c_s^2 kept between a quarter of a cell and r_K/2
    (Sec. 3.1.1); distances and r_acc in cells (r_BH / dx).  Ratios to the
    host cell, from cell centres computed here."""
    params = syn.sink_params(r_K=4.0, gamma=2.0, G=0.01, dt=1e-9, rho_min=0.0)
    box = syn.Box((16, 16, 16), 4)
    state = syn.uniform_gas(box, 1.0, e_th=0.5)  # c_s = 1
    xs = np.array([8.3, 7.6, 8.45])
    sink = one(*xs, Gm / 0.01)
    r = orc.cycle(params, box, state, sink, dx=dx)
    assert r["counts"][0] == 0
    drho = box.valid(r["buf"])[0]
    k, j, i = np.nonzero(drho)
    d2 = np.sum((np.stack([i + 0.5, j + 0.5, k + 0.5], axis=1) - xs) ** 2, axis=1)
    assert np.all(d2 < 16.0)
    h = np.argmin(d2)
    want = np.exp(-(d2 - d2[h]) / (r_acc * r_acc))
    got = drho[k, j, i] / drho[k[h], j[h], i[h]]
    keep = want > 1e-250
    assert keep.sum() > 6
    assert np.allclose(got[keep], want[keep], rtol=1e-11, atol=0)


@pytest.mark.parametrize("dx", [1.0, 0.5])
def test_truelove_density_is_the_floor_of_accretion(orc, dx):
    """A sink whose Bondi rate is negligible, in uniform gas above the Truelove
    density rho_Tr = J^2 pi c_s^2 / (G dx^2) (Eq. truelove): the accretion
    rate that enforces the Truelove condition removes rho - rho_Tr from every
    kernel cell, which the 25% limiter lets through (Sec. 3.1.1), so every
    kernel cell ends at rho_Tr and every other cell keeps rho."""
    J, G, gamma = 0.25, 0.035, 5.0 / 3.0
    params = syn.sink_params(r_K=2.0, gamma=gamma, G=G, J=J, dt=1e-12, rho_min=0.0)
    box = syn.Box((8, 8, 8), 2)
    rho0 = 40.0
    state = syn.uniform_gas(box, rho0, e_th=0.9)  # c_s^2 = gamma (gamma - 1) e_th = 1
    cs2 = gamma * (gamma - 1.0) * 0.9
    rho_tr = J * J * math.pi * cs2 / (G * dx * dx)
    assert rho_tr < rho0 and rho0 - rho_tr > rho0 / 4
    xs = (4.2, 3.7, 4.6)
    r = orc.cycle(params, box, state, one(*xs, 1.0), dx=dx)
    rho = box.valid(state)[0]
    k, j, i = np.indices(rho.shape)
    d2 = (i + 0.5 - xs[0]) ** 2 + (j + 0.5 - xs[1]) ** 2 + (k + 0.5 - xs[2]) ** 2
    inside = d2 < 4.0
    assert inside.sum() > 20
    assert np.allclose(rho[inside], rho_tr, rtol=1e-13, atol=0)
    assert np.all(rho[~inside] == rho0)
    assert r["counts"][0] == 0


def test_bondi_hoyle_depends_on_the_relative_velocity(orc):
    """Eq. mdot uses the gas velocity relative to the sink: a sink moving at
    -v through gas at rest accretes as a sink at rest in gas moving at v, and,
    the swallowed gas being at rest, keeps its momentum."""
    G, m, dt = 0.01, 10.0, 1e-3
    vel = np.array([0.25, -0.5, 1.25])
    params = syn.sink_params(r_K=4.0, gamma=2.0, G=G, dt=dt, rho_min=0.0)
    box = syn.Box((16, 16, 16), 4)
    state = syn.uniform_gas(box, 1.0, e_th=0.5)
    sink = one(8.3, 7.6, 8.45, m, p=tuple(-m * vel))
    r = orc.cycle(params, box, state, sink)
    assert r["counts"][0] == 0
    v2 = float(vel @ vel)
    lam = math.exp(1.5) / 4.0
    mdot = 4.0 * math.pi * G * G * m * m * math.sqrt((lam * lam + v2) / (1.0 + v2) ** 4)
    assert sink["m"][0] - m == pytest.approx(mdot * dt, rel=1e-13)
    for a, k in enumerate(("px", "py", "pz")):
        assert sink[k][0] == -m * vel[a]


@pytest.mark.parametrize("vel,dx,rho0", [((0.0, 0.0, 0.0), 1.0, 1.0), ((0.25, -0.5, 1.25), 1.0, 1.0),
                                         ((0.25, -0.5, 1.25), 0.5, 1.0), ((0.0, 0.0, 0.0), 1.0, 2.5)])
def test_bondi_hoyle_closed_form(orc, vel, dx, rho0):
    """Uniform gas (rho0, c_s = 1 exactly with gamma = 2 and e_th = 1/2)
    moving at vel past a sink at rest: the accreted mass over dt is the first
    line of Eq. mdot, 4 pi rho0 G^2 m^2 sqrt((lambda^2 c^2 + v^2)/(c^2 + v^2)^4)
    dt, because the normalised weights of Eq. kernel_wgt sum to 1 and neither
    the Truelove branch nor the limiter is active."""
    G, m, dt = 0.01, 10.0, 1e-3
    params = syn.sink_params(r_K=4.0, gamma=2.0, G=G, dt=dt, rho_min=0.0)
    box = syn.Box((16, 16, 16), 4)
    state = syn.uniform_gas(box, rho0, vel=vel, e_th=0.5)
    sink = one(8.3, 7.6, 8.45, m)
    old = state.copy()
    r = orc.cycle(params, box, state, sink, dx=dx)
    assert r["counts"][0] == 0
    v2 = vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2
    lam = math.exp(1.5) / 4.0
    mdot = 4.0 * math.pi * rho0 * G * G * m * m * math.sqrt((lam * lam + v2) / (1.0 + v2) ** 4)
    dm = sink["m"][0] - m
    assert dm == pytest.approx(mdot * dt, rel=1e-13)
    dgas = math.fsum((box.valid(state)[0] - box.valid(old)[0]).ravel()) * dx ** 3
    assert dgas == pytest.approx(-mdot * dt, rel=1e-10)
    # the sink keeps the momentum of the gas it swallowed (Eq. accretion_function row 2)
    for a in range(3):
        assert sink[("px", "py", "pz")[a]][0] == pytest.approx(vel[a] * mdot * dt, rel=1e-12, abs=1e-20)


# --------------------------------------------------------------------------
# conservation (Eq. conservation; "manifestly" conservative Step 5)
# --------------------------------------------------------------------------

def _fb_cloud(rng, box, count):
    x = rng.uniform(0, box.n[0], count)
    y = rng.uniform(0, box.n[1], count)
    z = rng.uniform(0, box.n[2], count)
    m = np.exp(rng.uniform(math.log(1e-3), math.log(1e-1), count))
    v = rng.normal(0, 0.1, (3, count))
    return dict(x=x, y=y, z=z, m=m, px=m * v[0], py=m * v[1], pz=m * v[2], e=np.ones(count))


def test_kernel_cut_at_a_non_periodic_face_keeps_the_ledger(orc):
    """On a non-periodic axis the kernel stops at the domain face (reading R2):
    no cell outside the domain is part of it, and the summed changes of the
    valid cells carry exactly the ejecta mass, momentum and energy (EJ
    regime), with nothing left in the buffer's ghost cells of that axis."""
    box = syn.Box((12, 12, 12), 3)
    rng = np.random.default_rng(17)
    state = syn.gas_state(rng, box)
    p = many([(0.3, 6.2, 5.7, 0.02, 0.001, -0.002, 0.0005, 1.0),
              (11.6, 0.4, 11.8, 0.05, -0.003, 0.001, 0.002, 1.0)])
    params = syn.feedback_params(A_sf=1e9)
    for s in range(2):
        ijk, _ = orc.kernel_of(params, box, p["x"][s], p["y"][s], p["z"][s], periodic=(0, 1, 1))
        assert np.all((ijk[:, 0] >= 0) & (ijk[:, 0] < 12))
        assert len(ijk) < len(orc.kernel_of(params, box, p["x"][s], p["y"][s], p["z"][s])[0])
    r = orc.cycle(params, box, state, p, periodic=(0, 1, 1))
    D = box.valid(r["buf"]).reshape(5, -1)
    assert math.fsum(D[0]) == pytest.approx(math.fsum(p["m"]), rel=1e-13)
    for a, k in enumerate(("px", "py", "pz")):
        assert math.fsum(D[1 + a]) == pytest.approx(math.fsum(p[k]), rel=1e-12)
    ekin = (p["px"] ** 2 + p["py"] ** 2 + p["pz"] ** 2) / (2 * p["m"])
    assert math.fsum(D[4]) == pytest.approx(math.fsum(p["e"] + ekin), rel=1e-13)
    g = box.grid(r["buf"])
    assert np.all(g[:, :, :, :3] == 0) and np.all(g[:, :, :, -3:] == 0)


@pytest.mark.parametrize("dx", [1.0, 0.5])
def test_feedback_conservation_ej_regime(orc, dx):
    """EJ regime (|p_radial| = 0, Eq. dp): the summed buffer times the cell
    volume V = dx^3 carries exactly the ejecta mass, the ejecta momentum and
    E_sn + E_kin (Eq. conservation), for any cell size."""
    rng = np.random.default_rng(3)
    box = syn.Box((16, 16, 16), 2)
    state = syn.gas_state(rng, box)
    parts = _fb_cloud(rng, box, 40)
    params = syn.feedback_params(A_sf=1e9)
    r = orc.cycle(params, box, state, parts, dx=dx)
    assert np.all(r["gathered"][11] == 0.0)  # every particle in EJ
    D = box.valid(r["buf"]).reshape(5, -1)
    V = dx ** 3
    assert math.fsum(D[0]) * V == pytest.approx(math.fsum(parts["m"]), rel=1e-13)
    for a, k in enumerate(("px", "py", "pz")):
        assert math.fsum(D[1 + a]) * V == pytest.approx(math.fsum(parts[k]), rel=1e-12, abs=1e-15)
    ekin = (parts["px"] ** 2 + parts["py"] ** 2 + parts["pz"] ** 2) / (2 * parts["m"])
    assert math.fsum(D[4]) * V == pytest.approx(math.fsum(parts["e"] + ekin), rel=1e-13)


@pytest.mark.parametrize("regime_Asf", [(1, 100.0), (2, 1e-3)])
def test_feedback_conservation_symmetric_kernel(orc, regime_Asf):
    """A particle exactly at a cell centre has a point-symmetric kernel, so the
    radial momenta cancel (Sec. 3.2.1) and the momentum and energy ledgers
    reduce to p_ej and E_sn + E_kin."""
    regime, A_sf = regime_Asf
    rng = np.random.default_rng(4)
    box = syn.Box((12, 12, 12), 2)
    state = syn.gas_state(rng, box)
    p = one(5.5, 6.5, 4.5, 0.05, p=(0.004, -0.003, 0.002))
    params = syn.feedback_params(A_sf=A_sf)
    r = orc.cycle(params, box, state, p)
    assert r["gathered"][11][0] == regime
    assert r["gathered"][7][0] > 0.0
    D = box.valid(r["buf"]).reshape(5, -1)
    scale = math.fsum(np.abs(D[1:4]).ravel())
    for a, k in enumerate(("px", "py", "pz")):
        assert abs(math.fsum(D[1 + a]) - p[k][0]) <= 1e-13 * scale
    ekin = (0.004 ** 2 + 0.003 ** 2 + 0.002 ** 2) / (2 * 0.05)
    assert math.fsum(D[4]) == pytest.approx(1.0 + ekin, rel=1e-13)
    assert math.fsum(D[0]) == pytest.approx(0.05, rel=1e-13)


def test_feedback_energy_ledger_single_particle(orc):
    """Single particle, any position: the energy row's cross term equals
    v_COM . (momentum deposited minus ejecta momentum), i.e. the rows of Eq. du
    are consistent, and total energy = E_sn + E_kin + v_COM . sum p_rad V."""
    rng = np.random.default_rng(5)
    box = syn.Box((12, 12, 12), 2)
    state = syn.gas_state(rng, box)
    p = one(5.27, 6.81, 4.05, 0.03, p=(0.003, -0.002, 0.001), e=1.0)
    r = orc.cycle(syn.feedback_params(), box, state, p)
    D = box.valid(r["buf"]).reshape(5, -1)
    G = r["gathered"][:, 0]
    prad_sum = np.array([math.fsum(D[1 + a]) - p[k][0] for a, k in enumerate(("px", "py", "pz"))])
    ekin = (0.003 ** 2 + 0.002 ** 2 + 0.001 ** 2) / (2 * 0.03)
    expect = 1.0 + ekin + float(np.dot(G[2:5], prad_sum))
    assert math.fsum(D[4]) == pytest.approx(expect, rel=1e-13)
    assert np.linalg.norm(prad_sum) <= G[7] * (1 + 1e-12)


def test_feedback_radial_momentum_magnitude(orc):
    """Gas and particle at rest: every cell receives only p_rad,c, whose
    magnitudes sum to |p_radial| (Sec. 3.2.1), and the energy is E_sn."""
    box = syn.Box((12, 12, 12), 2)
    state = syn.uniform_gas(box, 2.0, e_th=1e3)
    p = one(5.27, 6.81, 4.05, 0.03)
    r = orc.cycle(syn.feedback_params(), box, state, p)
    D = box.valid(r["buf"]).reshape(5, -1)
    mag = np.sqrt(D[1] ** 2 + D[2] ** 2 + D[3] ** 2)
    assert math.fsum(mag) == pytest.approx(r["gathered"][7][0], rel=1e-13)
    assert math.fsum(D[4]) == pytest.approx(1.0, rel=1e-14)


def test_feedback_radial_momentum_points_outward(orc):
    """Gas and particle at rest: the momentum each cell receives is the radial
    momentum of Sec. 3.2.1, so it points from the supernova to the cell's
    centre (collinear with x_c - x_s, positive projection).  The centres come
    from the cell indices here, not from the oracle's kernel enumeration."""
    box = syn.Box((12, 12, 12), 2)
    state = syn.uniform_gas(box, 2.0, e_th=1e3)
    xs = np.array([5.27, 6.81, 4.05])
    p = one(*xs, 0.03)
    r = orc.cycle(syn.feedback_params(), box, state, p)
    D = box.valid(r["buf"])  # [5][k][j][i]
    k, j, i = np.nonzero(np.sqrt(D[1] ** 2 + D[2] ** 2 + D[3] ** 2) > 0)
    assert i.size > 20
    d = np.stack([i + 0.5, j + 0.5, k + 0.5], axis=1) - xs
    dp = np.stack([D[1][k, j, i], D[2][k, j, i], D[3][k, j, i]], axis=1)
    dn = d / np.linalg.norm(d, axis=1)[:, None]
    along = np.sum(dp * dn, axis=1)
    assert np.all(along > 0)
    assert np.allclose(np.linalg.norm(dp - along[:, None] * dn, axis=1), 0.0, atol=1e-14 * along.max())


def test_supernova_energy_sums_to_prescribed_value(orc):
    """Gas at rest and ejecta at rest: v_COM = 0, so the deposited energy is
    exactly E_sn (Eq. du), whatever the limiter does to momentum."""
    rng = np.random.default_rng(6)
    box = syn.Box((16, 16, 16), 2)
    state = syn.gas_state(rng, box)
    v = box.valid(state)
    v[4] = v[0] * 1.0
    v[1:4] = 0.0
    parts = _fb_cloud(rng, box, 12)
    for k in ("px", "py", "pz"):
        parts[k][:] = 0.0
    parts["e"] = rng.uniform(0.5, 2.0, 12)
    old = state.copy()
    orc.cycle(syn.feedback_params(), box, state, parts)
    dE = math.fsum((box.valid(state)[4] - box.valid(old)[4]).ravel())
    assert dE == pytest.approx(math.fsum(parts["e"]), rel=1e-13)


def test_sink_conservation_with_active_limiter(orc):
    """Sinks on lognormal gas with the 25% cap active: gas mass and momentum
    lost equal what the sinks gain (Eq. conservation), through Step 4's
    limited return."""
    rng = np.random.default_rng(7)
    box = syn.Box((20, 20, 20), 4)
    state = syn.gas_state(rng, box)
    x = rng.uniform(0, 20, (3, 10))
    m = np.exp(rng.uniform(0, math.log(100), 10))
    vv = rng.normal(0, 0.1, (3, 10))
    sinks = dict(x=x[0].copy(), y=x[1].copy(), z=x[2].copy(), m=m.copy(), px=m * vv[0], py=m * vv[1],
                 pz=m * vv[2], e=np.zeros(10))
    old = state.copy()
    m0, p0 = sinks["m"].copy(), np.array([sinks[k].copy() for k in ("px", "py", "pz")])
    r = orc.cycle(syn.sink_params(dt=0.5), box, state, sinks, want_eta=True)
    assert r["counts"][0] > 0, "the limiter should be active somewhere"
    eta = r["eta"]
    D = box.valid(r["buf"]).reshape(5, -1)
    lim = [math.fsum(eta * D[f]) for f in range(5)]
    dm = math.fsum(sinks["m"] - m0)
    assert lim[0] + dm == pytest.approx(0.0, abs=1e-13 * dm)
    for a, k in enumerate(("px", "py", "pz")):
        dp = math.fsum(sinks[k] - p0[a])
        assert lim[1 + a] + dp == pytest.approx(0.0, abs=1e-13 * math.fsum(np.abs(eta * D[1 + a])))
    new, ov = box.valid(state).reshape(5, -1), box.valid(old).reshape(5, -1)
    assert np.all(np.abs(new - (ov + eta * D)) <= 4e-16 * np.abs(ov) + 1e-300)


# --------------------------------------------------------------------------
# limiters (Sec. 3.1.1 accretion limiter; Eq. lambda)
# --------------------------------------------------------------------------

def test_accretion_keeps_velocity_and_specific_energy(orc):
    """Eq. accretion_function removes gas at the cell's own velocity and
    specific energy (rows Delta rho (1, v, e_sp + v^2/2)), and one eta scales
    all rows, so every cell keeps p/rho and E/rho through a sink pass, to
    rounding, whether or not the limiter acts."""
    rng = np.random.default_rng(12)
    box = syn.Box((20, 20, 20), 4)
    state = syn.gas_state(rng, box, sigma_p=0.3)
    n = 10
    x = rng.uniform(0, 20, (3, n))
    m = np.exp(rng.uniform(0, math.log(100), n))
    sinks = dict(x=x[0].copy(), y=x[1].copy(), z=x[2].copy(), m=m, px=np.zeros(n), py=np.zeros(n),
                 pz=np.zeros(n), e=np.zeros(n))
    old = box.valid(state).reshape(5, -1).copy()
    r = orc.cycle(syn.sink_params(dt=5.0), box, state, sinks, want_eta=True)
    new = box.valid(state).reshape(5, -1)
    touched = new[0] != old[0]
    assert touched.sum() > 1000 and r["counts"][0] > 0
    for f in (1, 2, 3, 4):
        a, b = new[f][touched] / new[0][touched], old[f][touched] / old[0][touched]
        assert np.all(np.abs(a - b) <= 1e-12 * np.abs(b) + 1e-15), f


def test_sink_limiter_bounds(orc):
    """rho_new >= rho_min, rho_new >= min((1 - cap) rho, rho_Tr), eta in [0, 1]."""
    rng = np.random.default_rng(8)
    box = syn.Box((16, 16, 16), 4)
    state = syn.gas_state(rng, box)
    params = syn.sink_params(dt=5.0, rho_min=0.05)
    n = 24
    x = rng.uniform(0, 16, (3, n))
    m = np.exp(rng.uniform(0, math.log(100), n))
    sinks = dict(x=x[0].copy(), y=x[1].copy(), z=x[2].copy(), m=m, px=np.zeros(n), py=np.zeros(n), pz=np.zeros(n),
                 e=np.zeros(n))
    old = state.copy()
    r = orc.cycle(params, box, state, sinks, want_eta=True)
    rho, rho0 = box.valid(state)[0].ravel(), box.valid(old)[0].ravel()
    U = box.valid(old).reshape(5, -1)
    eint = np.maximum(U[4] - (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / (2 * U[0]), 0)
    cs2 = params["gamma"] * (params["gamma"] - 1) * eint / U[0]
    rho_tr = params["J"] ** 2 * math.pi * cs2 / params["G"]
    assert np.all(r["eta"] >= 0) and np.all(r["eta"] <= 1)
    assert r["counts"][0] > 0
    # removal is at most max(0, min(max(cap rho, rho - rho_Tr), rho - rho_min))
    floor = np.minimum(rho0, np.maximum(np.minimum((1 - params["cap"]) * rho0, rho_tr), params["rho_min"]))
    assert np.all(rho >= floor * (1 - 1e-14))
    # nothing that started above the floor ends below it
    assert np.all(rho[rho0 >= params["rho_min"]] >= params["rho_min"] * (1 - 1e-14))


def _apply_single_cell(orc, U, D, params):
    box = syn.Box((1, 1, 1), 0)
    st = box.empty(0.0)
    buf = box.empty(0.0)
    st[:, 0] = U
    buf[:, 0] = D
    eta, counts = orc.apply(params, box, st, buf, want_eta=True)
    return st[:, 0].copy(), eta[0], counts


def test_sn_lambda_closed_form_gas_at_rest(orc):
    """p = 0: the constraint of Eq. lambda gives lambda = sqrt(2 rho' (E' -
    e_int0 rho'/rho)) / |dp| when that is below 1."""
    rho, E = 1.3, 0.7
    D = np.array([0.2, 3.0, -4.0, 1.5, 0.9])
    U = np.array([rho, 0.0, 0.0, 0.0, E])
    new, lam, counts = _apply_single_cell(orc, U, D, syn.feedback_params())
    rho1, E1 = rho + D[0], E + D[4]
    expect = math.sqrt(2 * rho1 * (E1 - E * rho1 / rho)) / math.sqrt(D[1] ** 2 + D[2] ** 2 + D[3] ** 2)
    assert expect < 1
    assert lam == pytest.approx(expect, rel=1e-14)
    assert np.allclose(new[1:4], lam * D[1:4], rtol=1e-15, atol=0)
    assert counts[0] == 1


def test_sn_lambda_constraint_holds_after_limiting(orc):
    """Whenever a root exists, the limited state obeys Eq. lambda: the internal
    energy after deposit is at least e_int0 rho'/rho (to rounding), and lambda
    is the largest such value (the constraint is tight when lambda < 1)."""
    rng = np.random.default_rng(9)
    params = syn.feedback_params()
    seen = 0
    for _ in range(300):
        rho = math.exp(rng.normal(-0.5, 1))
        p = rng.normal(0, 0.3, 3)
        eint = rho * rng.uniform(0.01, 1.0)
        E = eint + p @ p / (2 * rho)
        D = np.concatenate([[rng.uniform(0, 0.1)], rng.normal(0, 1.0, 3), [rng.uniform(0, 0.5)]])
        U = np.concatenate([[rho], p, [E]])
        new, lam, counts = _apply_single_cell(orc, U, D, params)
        assert 0.0 <= lam <= 1.0
        rho1 = rho + D[0]
        bound = eint * rho1 / rho
        e_after = new[4] - (new[1:4] @ new[1:4]) / (2 * rho1)
        if counts[1] == 0:
            assert e_after >= bound - 1e-10 * (abs(new[4]) + abs(bound))
            if lam < 1:
                seen += 1
                assert e_after == pytest.approx(bound, rel=1e-8, abs=1e-10 * abs(new[4]))
    assert seen > 10


def _largest_feasible_lambda(U, D):
    """Brute force of Eq. lambda: the largest l in [0, 1] at which the internal
    energy after the deposit, with momentum change l dp, is at least
    e_int0 rho'/rho; found by a fine scan and bisection, with no quadratic
    formula.  None when no l in [0, 1] qualifies."""
    rho, p, E = U[0], U[1:4], U[4]
    rho1, E1 = rho + D[0], E + D[4]
    bound = (E - p @ p / (2 * rho)) * rho1 / rho

    def ok(lam):
        pn = p + lam * D[1:4]
        return E1 - pn @ pn / (2 * rho1) >= bound

    grid = np.linspace(0.0, 1.0, 200001)
    good = [lam for lam in grid[::-1] if ok(lam)][:1]
    if not good:
        return None
    lo = good[0]
    hi = min(1.0, lo + 1.0 / 200000)
    if ok(hi):
        return hi
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if ok(mid) else (lo, mid)
    return lo


@pytest.mark.parametrize("case", [
    # p . dp < 0 and the constraint failing at 0 and at 1: two roots in (0, 1)
    ([1.0, 1.0, 0.0, 0.0, 1.5], [0.1, -3.0, 0.0, 0.0, 0.05]),
    ([2.0, 0.5, -1.0, 0.3, 2.0], [0.05, -2.5, 3.0, -1.0, 0.02]),
    # one root in (0, 1)
    ([1.3, 0.2, 0.0, 0.0, 0.8], [0.2, 3.0, -4.0, 1.5, 0.9]),
])
def test_sn_lambda_is_the_largest_feasible_value(orc, case):
    """Eq. lambda keeps as much of the deposited momentum as the temperature
    constraint allows: lambda is the largest value in [0, 1] that satisfies
    it, here found by brute force."""
    U, D = np.array(case[0]), np.array(case[1])
    want = _largest_feasible_lambda(U, D)
    assert want is not None and want < 1.0
    _, lam, _ = _apply_single_cell(orc, U, D, syn.feedback_params())
    assert lam == pytest.approx(want, abs=1e-9)


@pytest.mark.parametrize("case", [
    # dp orthogonal to p: |p + l dp| >= |p| for every l, the quadratic has no real root
    ([1.0, 1.0, 0.0, 0.0, 1.0], [1.0, 0.0, 1.0, 0.0, 0.1]),
    # dp along p: both roots negative
    ([1.0, 1.0, 0.0, 0.0, 1.0], [1.0, 1.0, 0.0, 0.0, 0.1]),
    # a small dp against p: both roots above 1
    ([1.0, 1.0, 0.0, 0.0, 1.0], [1.0, -0.3, 0.0, 0.0, 0.1]),
])
def test_sn_lambda_without_a_feasible_value(orc, case):
    """Where no lambda in [0, 1] satisfies Eq. lambda (brute force), the
    momentum change is dropped (lambda = 0, the reading for that case) and the
    cell is counted; the mass and energy changes still go in."""
    U, D = np.array(case[0]), np.array(case[1])
    assert _largest_feasible_lambda(U, D) is None
    new, lam, counts = _apply_single_cell(orc, U, D, syn.feedback_params())
    assert lam == 0.0
    assert counts[1] == 1
    assert np.array_equal(new[1:4], U[1:4])
    assert new[0] == U[0] + D[0] and new[4] == U[4] + D[4]


# --------------------------------------------------------------------------
# regimes (Eq. dp, Eq. psnr)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("mu_H", [1.0, 1.4])
@pytest.mark.parametrize("target", [0.02, 0.5, 3.0])
def test_regime_and_radial_momentum(orc, target, mu_H):
    """Uniform density rho0 chosen so that R_M hits the target; |p_radial|
    must be 0 (EJ), sqrt(2 M_ej eps_K E_sn) (ST) or A_p n_H^-0.17 (MC), with
    n_H = M_snr / (mu_H V_snr) the hydrogen number density."""
    box = syn.Box((12, 12, 12), 2)
    params = syn.feedback_params(mu_H=mu_H)
    M_ej, E_sn = 0.01, 1.0
    pos = (5.3, 6.2, 4.7)
    # V_snr does not depend on the gas: read it once, then solve for rho0.
    probe = orc.gather(params, box, syn.uniform_gas(box, 1.0), one(*pos, M_ej, e=E_sn))
    Vsnr = probe[1][0]

    def R_M(rho0):
        M = rho0 * Vsnr + M_ej
        n = M / (mu_H * Vsnr)
        return M / (params["A_sf"] * n ** -0.26)

    lo, hi = 1e-6, 1e6
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if R_M(mid) < target:
            lo = mid
        else:
            hi = mid
    rho0 = math.sqrt(lo * hi)
    G = orc.gather(params, box, syn.uniform_gas(box, rho0), one(*pos, M_ej, e=E_sn))[:, 0]
    assert G[6] == pytest.approx(target, rel=1e-9)
    nH = (rho0 * Vsnr + M_ej) / (mu_H * Vsnr)
    assert G[5] == pytest.approx(nH, rel=1e-12)
    if target <= 0.027:
        assert G[11] == 0 and G[7] == 0.0
    elif target <= 1.0:
        assert G[11] == 1 and G[7] == pytest.approx(math.sqrt(2 * M_ej * 0.28 * E_sn), rel=1e-15)
    else:
        assert G[11] == 2 and G[7] == pytest.approx(params["A_p"] * nH ** -0.17, rel=1e-13)


def test_mc_kinetic_fraction_calibration():
    """Sec. 3.2.1: in MC the kinetic energy of the terminal momentum is
    4.6e50 erg = 0.46 E_sn.  With P_snr = 2.8e5 Msun km/s (Eq. psnr at n_H = 1)
    that figure is P_snr^2 / (2 M_sf) for the shell-formation mass
    M_sf(n_H = 1) = 1679 Msun; the code-unit A_p keeps the same ratio to
    A_sf = M_sf(1)."""
    msun, kms, esn = 1.98847e33, 1e5, 1e51
    p_snr = 2.8e5 * msun * kms
    assert p_snr ** 2 / (2 * 1679 * msun) / esn == pytest.approx(0.46, abs=0.005)
    fp = syn.feedback_params()
    assert fp["A_p"] ** 2 / (2 * fp["A_sf"]) == pytest.approx(0.46, rel=1e-12)


# --------------------------------------------------------------------------
# covered fraction omega: symmetry and limits
# --------------------------------------------------------------------------

def test_omega_is_one_for_topHat_and_interior_cells(orc):
    box = syn.Box((12, 12, 12), 2)
    ijk, om = orc.kernel_of(syn.feedback_params(subsample=1), box, 5.3, 6.1, 4.8)
    assert np.all(om == 1.0)
    ijk, om = orc.kernel_of(syn.feedback_params(subsample=4), box, 5.3, 6.1, 4.8)
    for (i, j, k), w in zip(ijk, om):
        far = 0.0
        for c, x in zip((i, j, k), (5.3, 6.1, 4.8)):
            far += max(abs(c - x), abs(c + 1 - x)) ** 2
        if far < 4.0:
            assert w == 1.0
        assert 0.0 < w <= 1.0 or w == 0.0


@pytest.mark.parametrize("pos", [(5.5, 6.5, 4.5), (5.0, 6.0, 4.0)])
def test_omega_reflection_symmetry(orc, pos):
    """A particle at a cell centre, or at a cell corner, sees a kernel whose
    covered fractions are symmetric under reflection through the particle in
    each axis (an off-by-half sub-point placement breaks this)."""
    box = syn.Box((12, 12, 12), 2)
    ijk, om = orc.kernel_of(syn.feedback_params(subsample=4), box, *pos)
    d = {tuple(c): w for c, w in zip(ijk, om)}
    for (i, j, k), w in d.items():
        for a in range(3):
            c = [i, j, k]
            # reflection of cell index c about position x: c' = 2x - 1 - c
            c[a] = int(round(2 * pos[a] - 1 - c[a]))
            assert d.get(tuple(c)) == w


def test_omega_converges_to_covered_volume(orc):
    """Sum of omega over the kernel tends to the volume of the union of member
    cells intersected with the sphere; checked against a 64^3-per-cell
    midpoint estimate made here, at S = 16 (error O(1/S))."""
    box = syn.Box((12, 12, 12), 2)
    pos = np.array([5.31, 6.14, 4.77])
    ijk, om = orc.kernel_of(syn.feedback_params(subsample=16), box, *pos)
    t = (np.arange(64) + 0.5) / 64
    X, Y, Z = np.meshgrid(t, t, t, indexing="ij")
    for (i, j, k), w in zip(ijk, om):
        d2 = (i + X - pos[0]) ** 2 + (j + Y - pos[1]) ** 2 + (k + Z - pos[2]) ** 2
        frac = np.count_nonzero(d2 < 4.0) / 64 ** 3
        assert abs(w - frac) < 0.06


# --------------------------------------------------------------------------
# brute force on tiny boxes: kernel membership, ghost mapping and Step 2
# --------------------------------------------------------------------------

@pytest.mark.parametrize("rK", [1.0, 2.0, 3.0, 4.0])
def test_membership_ties_are_outside(orc, rK):
    """A particle on a cell centre puts cell centres at exactly r_K: those are
    outside the kernel (the strict "< r_K" of Sec. 3.2.1), as a scan of the
    whole box finds.  Particles on a face and on a corner are checked too."""
    box = syn.Box((12, 12, 12), 4)
    params = syn.feedback_params(r_K=rK, subsample=2)
    for x, y, z in ((5.5, 6.5, 4.5), (5.0, 6.5, 4.5), (6.0, 6.0, 6.0)):
        ijk, _ = orc.kernel_of(params, box, x, y, z)
        want = brute_members(box, x, y, z, rK)
        assert {tuple(c) for c in ijk} == want
        if x == 5.5:  # on a centre, the centres (r_K, 0, 0) away sit exactly at r_K
            assert [c for c in brute_members(box, x, y, z, rK + 1e-9) if c not in want]


@pytest.mark.parametrize("rK", [1.7, 2.7, 3.6])
def test_membership_reaches_ceil_rK_cells_away(orc, rK):
    """With a fractional part of r_K above 1/2, a cell ceil(r_K) cells from the
    host cell can be inside the kernel: offset o qualifies along x when
    o + 1/2 - f < r_K, f the particle's position within its cell.  A particle
    at f = 0.95 (y, z on centres) reaches it on the +x side, as a scan of the
    whole box finds."""
    box = syn.Box((12, 12, 12), 4)
    params = syn.feedback_params(r_K=rK, subsample=2)
    x, y, z = 5.95, 6.5, 4.5
    ijk, _ = orc.kernel_of(params, box, x, y, z)
    want = brute_members(box, x, y, z, rK)
    assert {tuple(c) for c in ijk} == want
    assert (5 + math.ceil(rK), 6, 4) in want


# r_K = 2.7: cells ceil(r_K) away can lie inside (an offset o qualifies when
# o < r_K - 1/2 + f, f the position within the host cell), which half-integer
# radii never show
@pytest.mark.parametrize("n,g,rK,seed", [(5, 2, 2.0, 1), (4, 3, 2.5, 2), (7, 4, 4.0, 3), (6, 2, 1.5, 4),
                                         (5, 3, 2.7, 5)])
def test_membership_and_fold_brute_force(orc, n, g, rK, seed):
    """Every (particle, buffer cell) pair found by scanning the whole padded
    box equals the oracle's kernel; after Step 2 every valid cell holds the sum
    of all pairs whose buffer cell is one of its periodic images."""
    rng = np.random.default_rng(seed)
    box = syn.Box((n, n + 1, n - 1), g)
    params = syn.feedback_params(r_K=rK, subsample=2)
    state = syn.gas_state(rng, box)
    parts = _fb_cloud(rng, box, 3)
    for s in range(3):
        ijk, _ = orc.kernel_of(params, box, parts["x"][s], parts["y"][s], parts["z"][s])
        assert {tuple(c) for c in ijk} == brute_members(box, parts["x"][s], parts["y"][s], parts["z"][s], rK)
    G = orc.gather(params, box, state, parts)
    singles = []
    for s in range(3):
        b = box.empty(0.0)
        sub = {k: v[s:s + 1].copy() for k, v in parts.items()}
        orc.deposit(params, box, state, sub, G[:, s:s + 1].copy(), b)
        singles.append(box.grid(b))
    buf = box.empty(0.0)
    orc.deposit(params, box, state, parts, G, buf)
    orc.fold(box, buf)
    valid = box.valid(buf)
    nx, ny, nz = box.n
    expect = np.zeros_like(valid)
    for s in range(3):
        gsum = singles[s]
        for k in range(-g, nz + g):
            for j in range(-g, ny + g):
                for i in range(-g, nx + g):
                    expect[:, k % nz, j % ny, i % nx] += gsum[:, k + g, j + g, i + g]
    assert np.allclose(valid, expect, rtol=1e-13, atol=1e-16)


def test_particle_order_independence(orc):
    """Sec. 3.2.1 / Sec. 2.2: the result does not depend on particle order up to
    floating-point rounding: |difference| <= n eps A_c per cell."""
    w = syn.make_workload("c1_32")
    box = w["box"]
    rng = np.random.default_rng(10)
    perm = rng.permutation(len(w["fb"]["x"]))
    a = w["state"].copy()
    b = w["state"].copy()
    ra = orc.cycle(w["fb_params"], box, a, w["fb"], want_abs=True)
    pb = {k: np.ascontiguousarray(v[perm]) for k, v in w["fb"].items()}
    rb = orc.cycle(w["fb_params"], box, b, pb)
    A = box.valid(ra["absbuf"])
    n = len(perm)
    assert np.all(np.abs(box.valid(ra["buf"]) - box.valid(rb["buf"])) <= n * 2.3e-16 * A)
    assert np.allclose(box.valid(a), box.valid(b), rtol=1e-13, atol=1e-15)


def test_state_ghost_cells_are_never_read(orc):
    """Ghosts of the state hold NaN in every workload; outputs stay finite."""
    w = syn.make_workload("c1_32")
    st = w["state"]
    orc.cycle(w["fb_params"], w["box"], st, w["fb"])
    orc.cycle(w["sink_params"], w["box"], st, w["sink"])
    assert np.all(np.isfinite(w["box"].valid(st)))
    assert np.all(np.isfinite(w["sink"]["m"]))


def test_cells_without_change_keep_their_bits(orc):
    """Step 5 adds eta * Delta U^sum: a cell whose summed change is zero in
    every field is left exactly as it was (a -0 momentum stays -0)."""
    box = syn.Box((8, 8, 8), 2)
    state = syn.uniform_gas(box, 1.0)
    v = box.valid(state)
    v[1] = -0.0
    v[4] = 1.0
    one = {"x": np.array([1.5]), "y": np.array([1.5]), "z": np.array([1.5]), "m": np.array([0.01]),
           "px": np.array([0.0]), "py": np.array([0.0]), "pz": np.array([0.0]), "e": np.array([1.0])}
    s = state.copy()
    orc.cycle(syn.feedback_params(r_K=1.0), box, s, one)
    far = box.valid(s)[:, 6, 6, 6]
    assert np.signbit(far[1]) and far[1] == 0.0
    assert box.valid(s)[0, 1, 1, 1] > 1.0


# --------------------------------------------------------------------------
# the plan's fixed slots: every kernel fits the per-particle bound C
# --------------------------------------------------------------------------

def _slot_bound(rK):
    """Offsets o whose cell centre can come strictly within r_K of some point
    of the host cell [0, 1)^3: the nearest such point is min(max(o + 1/2,
    0), 1) per axis, so the distance is max(|o| - 1/2, 0) per axis."""
    R = math.ceil(rK)
    n = 0
    for oz in range(-R, R + 1):
        for oy in range(-R, R + 1):
            for ox in range(-R, R + 1):
                d2 = sum(max(abs(o) - 0.5, 0.0) ** 2 for o in (ox, oy, oz))
                n += d2 < rK * rK
    return n


@pytest.mark.parametrize("rK,C", [(2.0, 81), (4.0, 461), (1.0, 27), (2.5, 117), (3.0, 251)])
def test_every_kernel_fits_the_slot_bound(orc, rK, C):
    """The workspace gives each particle C slots (81 at r_K = 2, 461 at
    r_K = 4), the number of offsets whose centre can come within r_K of the
    host cell: no position has more kernel cells, and the kernels of the
    positions at the host cell's corners, edge and face midpoints (where each
    offset's nearest point lies) cover exactly those C offsets."""
    bound = _slot_bound(rK)
    assert bound == C
    box = syn.Box((24, 24, 24), 6)
    params = syn.feedback_params(r_K=rK, subsample=1)
    rng = np.random.default_rng(int(rK * 8))
    eps = 1e-9
    ends = (eps, 0.5, 1.0 - eps)
    pos = [np.array([10.0 + a, 10.0 + b, 10.0 + c]) for a in ends for b in ends for c in ends]
    pos += list(rng.uniform(10.0, 11.0, (200, 3)))
    most, union = 0, set()
    for x, y, z in pos:
        ijk, _ = orc.kernel_of(params, box, float(x), float(y), float(z))
        most = max(most, len(ijk))
        union |= {(int(i) - 10, int(j) - 10, int(k) - 10) for i, j, k in ijk}
    assert most <= bound
    assert len(union) == bound
