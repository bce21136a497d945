"""Pins of the oracle's batched form (patches of one level tiling a periodic
domain; Sec. 2.2 Steps 1-5 with the ghost summation of App. A.2 across
patches).

- one patch whose 26 neighbours are itself is a periodic box: the batched
  oracle must give the single-box oracle's bits;
- the batched fold is the transpose of the ghost fill (each ghost cell is the
  image of exactly the cell it stands for), exactly on integer data;
- cutting a periodic box into uneven patches changes nothing but the order
  of the ghost sums: gathered rows are bit-identical, folded sums and the
  updated state agree within the summation-order bound, particles sitting on
  patch faces, edges and corners included;
- conservation of the injected mass and energy over the whole batch.
"""
import math

import numpy as np
import pytest

from paper_2509_18261_gb300 import synthetic as syn
from helpers import assert_bits_equal

FIELDS = ("x", "y", "z", "m", "px", "py", "pz", "e")


def _single_patch(n, g):
    b = syn.Batch(((n[0],), (n[1],), (n[2],)), g)
    assert np.all(b.nb == 0)
    return b


@pytest.mark.parametrize("kind", ["feedback", "sink"])
def test_single_patch_is_the_periodic_box(orc, kind):
    rng = np.random.default_rng(101)
    n = (16, 20, 12)
    box = syn.Box(n, 4)
    batch = _single_patch(n, 4)
    state = syn.gas_state(rng, box)
    parts = syn.particles(rng, n, 40, kind, clustered=16, nclusters=2)
    params = syn.feedback_params() if kind == "feedback" else syn.sink_params(dt=2.0)
    s_box, p_box = state.copy(), {k: v.copy() for k, v in parts.items()}
    ref = orc.cycle(params, box, s_box, p_box, want_abs=True, want_eta=True)
    arena = state.reshape(-1).copy()
    p_bat = {k: v.copy() for k, v in parts.items()}
    first = np.array([0, len(parts["x"])], dtype=np.int64)
    got = orc.batch_cycle(params, batch, arena, p_bat, first, want_abs=True, want_eta=True)
    assert_bits_equal(got["gathered"], ref["gathered"], "gathered")
    assert_bits_equal(box.valid(got["buf"].reshape(5, -1)), box.valid(ref["buf"]), "folded buffer")
    assert_bits_equal(box.valid(arena.reshape(5, -1)), box.valid(s_box), "state")
    assert_bits_equal(got["eta"], ref["eta"], "eta")
    for k in ("m", "px", "py", "pz"):
        assert_bits_equal(p_bat[k], p_box[k], k)
    assert np.array_equal(got["counts"], ref["counts"])
    if kind == "sink":
        assert ref["counts"][0] > 0, "the case should exercise the limiter"


@pytest.mark.parametrize("edges", [((16, 24, 16), (16, 24), (16, 16)), ((16, 16), (24,), (16, 16, 16))])
def test_fold_is_the_transpose_of_the_ghost_fill(orc, edges):
    rng = np.random.default_rng(7)
    batch = syn.Batch(edges, 4)
    B = rng.integers(-8, 9, batch.arena_len).astype(np.float64)
    V = batch.empty(0.0)
    for p in range(batch.np):
        batch.valid(V, p)[...] = rng.integers(-8, 9, batch.valid(V, p).shape)
    FB = B.copy()
    orc.batch_fold(batch, FB)
    FV = V.copy()
    orc.batch_fill_ghosts(batch, FV)
    lhs = sum(float(np.sum(batch.valid(FB, p) * batch.valid(V, p))) for p in range(batch.np))
    rhs = sum(float(np.sum(batch.grid(B, p) * batch.grid(FV, p))) for p in range(batch.np))
    assert lhs == rhs
    # and the fill copies the owner's values: global periodic wrap of the assembly
    G = batch.to_global(V)
    for p in range(batch.np):
        (x0, y0, z0), g = batch.origin[p], batch.g
        nx, ny, nz = batch.dims[p]
        Nx, Ny, Nz = batch.global_n
        ix = np.arange(x0 - g, x0 + nx + g) % Nx
        iy = np.arange(y0 - g, y0 + ny + g) % Ny
        iz = np.arange(z0 - g, z0 + nz + g) % Nz
        assert np.array_equal(batch.grid(FV, p), G[:, iz][:, :, iy][:, :, :, ix])


def _boundary_particles(rng, batch, kind, count):
    """Global positions within a cell of patch faces, edges and corners."""
    starts = [np.concatenate([[0], np.cumsum(e)]) for e in batch.edges]
    pos = np.empty((3, count))
    for a in range(3):
        N = batch.global_n[a]
        b = rng.choice(starts[a], count)
        off = rng.choice([-0.999, -0.5, -1e-9, 0.0, 1e-9, 0.5, 0.999], count)
        near = rng.random(count) < 0.8  # most particles sit on a boundary on this axis
        v = np.where(near, b + off, rng.random(count) * N)
        pos[a] = np.minimum(np.mod(v, N), np.nextafter(float(N), 0.0))
    p = syn.particles(rng, batch.global_n, count, kind)
    p["x"], p["y"], p["z"] = pos[0].copy(), pos[1].copy(), pos[2].copy()
    return p


def _to_patches(batch, parts):
    """Patch of each particle, local coordinates (exact: integer shifts), and
    the particles reordered patch after patch (stable)."""
    pid = np.zeros(len(parts["x"]), dtype=np.int64)
    local = {}
    idx = []
    for a, k in enumerate(("x", "y", "z")):
        starts = np.concatenate([[0], np.cumsum(batch.edges[a])])
        I = np.searchsorted(starts, parts[k], side="right") - 1
        idx.append(I)
        local[k] = parts[k] - starts[I]
    P0, P1, _ = batch.sgrid
    pid = (idx[2] * P1 + idx[1]) * P0 + idx[0]
    order = np.argsort(pid, kind="stable")
    out = {k: np.ascontiguousarray(parts[k][order]) for k in FIELDS}
    for k in ("x", "y", "z"):
        out[k] = np.ascontiguousarray(local[k][order])
    first = np.searchsorted(pid[order], np.arange(batch.np + 1)).astype(np.int64)
    return out, first, order


@pytest.mark.parametrize("kind", ["feedback", "sink"])
def test_decomposition_matches_the_global_box(orc, kind):
    rng = np.random.default_rng(202 if kind == "feedback" else 203)
    batch = syn.Batch(((16, 24, 16), (16, 24), (16, 24)), 4)
    gbox = syn.Box(batch.global_n, 4)
    gstate = syn.gas_state(rng, gbox)
    parts = _boundary_particles(rng, batch, kind, 120)
    params = syn.feedback_params() if kind == "feedback" else syn.sink_params(dt=2.0)
    gs, gp = gstate.copy(), {k: v.copy() for k, v in parts.items()}
    ref = orc.cycle(params, gbox, gs, gp, want_abs=True, want_eta=True)

    lp, first, order = _to_patches(batch, parts)
    pid = np.searchsorted(first, np.arange(len(order)), side="right") - 1
    for a, k in enumerate(("x", "y", "z")):
        assert np.all(lp[k] >= 0.0) and np.all(lp[k] < batch.dims[pid, a])
    arena = batch.from_global(gbox.valid(gstate))
    got = orc.batch_cycle(params, batch, arena, lp, first, want_abs=True, want_eta=True)

    # Step 1 gathers read the same cells in the same order
    assert_bits_equal(got["gathered"], ref["gathered"][:, order], "gathered")
    # Step 2: same terms, another order
    D_b = batch.to_global(got["buf"])
    D_g = gbox.valid(ref["buf"])
    A = gbox.valid(ref["absbuf"])
    assert np.all(np.abs(D_b - D_g) <= 1e-12 * A)
    touched = A[0] > 0
    assert touched.sum() > 1000
    # owner cells fed from several patches exist (faces, edges and corners)
    U_b = batch.to_global(arena)
    U_g = gbox.valid(gs)
    # eta, patch after patch, placed on the global grid
    eta_arena = batch.empty(0.0)
    for p in range(batch.np):
        nx, ny, nz = batch.dims[p]
        batch.valid(eta_arena, p)[0] = got["eta"][batch.vbase[p]:batch.vbase[p + 1]].reshape(nz, ny, nx)
    eta_glob = batch.to_global(eta_arena)[0]
    eta_ref = ref["eta"].reshape(gbox.n[::-1])
    assert np.all(np.abs(eta_glob - eta_ref) <= 1e-9)
    same = (eta_glob == 1.0) & (eta_ref == 1.0)
    assert np.all(np.abs(U_b - U_g)[:, same] <= 1e-12 * (np.abs(U_g) + A)[:, same])
    assert int(got["counts"][0]) == int(ref["counts"][0])
    if kind == "sink":
        assert ref["counts"][0] > 0
        for k in ("m", "px", "py", "pz"):
            d0 = parts[k][order]
            ref_d = gp[k][order] - d0
            got_d = lp[k] - d0
            assert np.all(np.abs(got_d - ref_d) <= 1e-10 * np.abs(ref_d) + 1e-15 * np.abs(d0))


def test_batch_feedback_conserves_mass_momentum_and_energy(orc):
    w = syn.make_batch_workload(supergrid=(3, 2, 2), edges=(16, 24), xmax=2000.0, seed=7)
    batch, state, parts, first = w["batch"], w["state"], w["fb"], w["fb_first"]
    assert first[-1] > 50
    params = syn.feedback_params(A_sf=1e6)  # EJ regime everywhere: no radial momentum
    old = state.copy()
    r = orc.batch_cycle(params, batch, state, {k: v.copy() for k, v in parts.items()}, first, want_abs=True)

    def total(arena, f, minus=None):
        return math.fsum(np.concatenate([
            (batch.valid(arena, p)[f] - (0.0 if minus is None else batch.valid(minus, p)[f])).ravel()
            for p in range(batch.np)]))

    ekin = (parts["px"] ** 2 + parts["py"] ** 2 + parts["pz"] ** 2) / (2.0 * parts["m"])
    # the folded sums (V = 1) hold exactly what the particles inject
    assert total(r["buf"], 0) == pytest.approx(math.fsum(parts["m"]), rel=1e-13)
    assert total(r["buf"], 4) == pytest.approx(math.fsum(parts["e"] + ekin), rel=1e-13)
    for a, k in enumerate(("px", "py", "pz")):
        assert abs(total(r["buf"], 1 + a) - math.fsum(parts[k])) <= 1e-13 * total(r["absbuf"], 1 + a)
    # the limiter scales momentum only: mass and energy reach the state in full
    assert total(state, 0, old) == pytest.approx(math.fsum(parts["m"]), rel=1e-12)
    assert total(state, 4, old) == pytest.approx(math.fsum(parts["e"] + ekin), rel=1e-12)


def test_batch_ghost_cells_of_the_state_are_never_read(orc):
    w = syn.make_batch_workload(supergrid=(3, 2, 2), edges=(16,), xmax=2000.0, seed=7)
    batch, parts, first = w["batch"], w["sink"], w["sink_first"]
    if first[-1] == 0:
        parts, first = w["fb"], w["fb_first"]
    params = syn.sink_params() if parts is w["sink"] else syn.feedback_params()
    a = w["state"].copy()
    b = w["state"].copy()
    for p in range(batch.np):  # different garbage in the ghosts
        gb = batch.grid(b, p)
        mask = np.ones(gb.shape[1:], dtype=bool)
        g = batch.g
        mask[g:-g, g:-g, g:-g] = False
        gb[:, mask] = 1e300
    ra = orc.batch_cycle(params, batch, a, {k: v.copy() for k, v in parts.items()}, first)
    rb = orc.batch_cycle(params, batch, b, {k: v.copy() for k, v in parts.items()}, first)
    assert_bits_equal(ra["gathered"], rb["gathered"], "gathered")
    for p in range(batch.np):
        assert_bits_equal(batch.valid(a, p), batch.valid(b, p), f"patch {p}")
