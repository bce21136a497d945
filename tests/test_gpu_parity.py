"""GPU path against the oracle, element by element, through the C ABI.

Sorted mode: bit-exact (gathered rows, buffer before and after Step 2, state
after Step 5, eta, sink particles).  Atomic mode: gathered rows bit-exact;
buffer within 1e-12 * A_c per cell and field, A_c = sum over contributions
of |Delta U^s_c| (the additions differ only in order); the state after Step
5 and the sinks after Step 4 within the bounds that buffer difference
implies through the limiters (tests/bounds.py).  "atomic" runs gather
and deposit through pmp_gather_deposit (one kernel for supernovae),
"atomic-split" through pmp_gather and pmp_deposit.
"""
import math

import numpy as np
import pytest

from paper_2509_18261_gb300 import synthetic as syn
from helpers import (assert_bits_equal, assert_state_within_bound, assert_within_abs, gpu_pass, oracle_pass,
                     sink_return_bound, valid_flat)

pytestmark = pytest.mark.gpu


def _check_pass(orc, params, box, state, parts, mode, periodic=(1, 1, 1), dx=1.0):
    ref = oracle_pass(orc, params, box, state, parts, periodic=periodic, dx=dx)
    g_dep = gpu_pass(params, box, state, parts, mode=mode, periodic=periodic, dx=dx, stop_after="deposit")
    g_fold = gpu_pass(params, box, state, parts, mode=mode, periodic=periodic, dx=dx, stop_after="fold")
    g = gpu_pass(params, box, state, parts, mode=mode, periodic=periodic, dx=dx)
    assert g["error"] == (0, -1), g["error"]
    have = parts is not None and parts["x"].size > 0
    if have:
        assert_bits_equal(g["gathered"], ref["gathered"], "gathered rows")
    # touched cells: exactly the oracle's (density rows are one-signed per kind)
    gb, rb = box.grid(g_dep["buf"]), box.grid(ref["pre_fold"])
    assert np.array_equal(gb[0] != 0.0, rb[0] != 0.0), "touched-cell set"
    if mode == "sorted":
        assert_bits_equal(gb, rb, "buffer after Step 1")
        assert_bits_equal(valid_flat(box, g_fold["buf"]), valid_flat(box, ref["buf"]), "buffer after Step 2")
        assert_bits_equal(valid_flat(box, g["state"]), valid_flat(box, ref["state"]), "state after Step 5")
        assert_bits_equal(g["eta"], ref["eta"], "eta")
        if have and params["kind"] == "sink":
            for k in ("m", "px", "py", "pz"):
                assert_bits_equal(g["parts"][k], ref["parts"][k], f"sink {k} after Step 4")
    else:
        A = valid_flat(box, ref["absbuf"])
        D = valid_flat(box, ref["buf"])
        assert_within_abs(valid_flat(box, g_fold["buf"]), D, A, "buffer after Step 2")
        assert_state_within_bound(params, valid_flat(box, state), D, A, ref["eta"], valid_flat(box, g["state"]),
                                  valid_flat(box, ref["state"]))
        if have and params["kind"] == "sink":
            for k in ("m", "px", "py", "pz"):
                a, b = g["parts"][k], ref["parts"][k]
                tol = sink_return_bound(params, box, state, parts, ref["parts"], k)
                assert np.all(np.abs(a - b) <= tol), (k, np.max(np.abs(a - b) / tol))
    assert g["counts"][0] == ref["counts"][0] or mode.startswith("atomic")
    return g, ref


@pytest.mark.parametrize("mode", ["sorted", "atomic", "atomic-split"])
def test_c1_feedback_then_sinks(orc, mode):
    """32^3 box, 4 ghosts: 64 supernovae then 8 sinks on the updated state
    (the two kinds are separate passes sharing the mesh)."""
    w = syn.make_workload("c1_32")
    box = w["box"]
    g, ref = _check_pass(orc, w["fb_params"], box, w["state"], w["fb"], mode)
    state2 = ref["state"]  # the oracle's post-feedback state feeds both sides
    _check_pass(orc, w["sink_params"], box, state2, w["sink"], mode)


def _cloud(rng, n, count, edge=True):
    x = [rng.uniform(0, n[a], count) for a in range(3)]
    if edge and count >= 6:
        x[0][0], x[1][0], x[2][0] = 0.0, 0.0, 0.0
        x[0][1] = np.nextafter(float(n[0]), 0.0)
        x[1][2], x[2][2] = 1.0, float(n[2] // 2)
        x[0][3], x[1][3], x[2][3] = 0.5, 1.5, 2.5
    m = np.exp(rng.uniform(math.log(1e-3), math.log(1e-1), count))
    v = rng.normal(0, 0.1, (3, count))
    return dict(x=x[0], y=x[1], z=x[2], m=m, px=m * v[0], py=m * v[1], pz=m * v[2], e=np.ones(count))


@pytest.mark.parametrize("mode", ["sorted", "atomic", "atomic-split"])
@pytest.mark.parametrize(
    "n,g,rK,S,periodic",
    [
        ((5, 6, 4), 2, 2.0, 4, (1, 1, 1)),
        ((7, 7, 7), 3, 2.5, 3, (1, 1, 1)),
        ((6, 5, 9), 2, 1.0, 1, (1, 1, 1)),
        ((8, 6, 7), 2, 1.5, 2, (1, 0, 1)),
        ((4, 4, 4), 4, 4.0, 8, (1, 1, 1)),
        ((9, 4, 5), 3, 3.0, 4, (0, 0, 0)),
    ],
)
def test_feedback_edge_boxes(orc, mode, n, g, rK, S, periodic):
    rng = np.random.default_rng(hash((n, g, rK, S)) % 2**32)
    box = syn.Box(n, g)
    state = syn.gas_state(rng, box)
    parts = _cloud(rng, n, 12)
    _check_pass(orc, syn.feedback_params(r_K=rK, subsample=S), box, state, parts, mode, periodic=periodic)


@pytest.mark.parametrize("mode", ["sorted", "atomic", "atomic-split"])
@pytest.mark.parametrize("n,g,rK,periodic,dt", [((9, 8, 10), 4, 4.0, (1, 1, 1), 0.5), ((7, 9, 6), 3, 2.7, (1, 0, 1), 2.0)])
def test_sink_edge_boxes(orc, mode, n, g, rK, periodic, dt):
    rng = np.random.default_rng(7 + g)
    box = syn.Box(n, g)
    state = syn.gas_state(rng, box)
    v = box.valid(state)
    v[0] *= 3.0  # denser gas: the Truelove branch and the 25% cap both engage
    v[4] *= 3.0
    parts = _cloud(rng, n, 10)
    parts["m"] = np.exp(rng.uniform(0, math.log(100), 10))
    _, ref = _check_pass(orc, syn.sink_params(r_K=rK, dt=dt), box, state, parts, mode, periodic=periodic)
    assert ref["counts"][0] > 0


def lambda_case_cells():
    """A 4 x 2 x 1 box whose first cells hold Eq. lambda's hard cases: three
    cells where no lambda in [0, 1] satisfies the constraint (no real root;
    both roots below 0; both above 1), one limited cell (one root in (0, 1)),
    one change without momentum; the rest of the buffer is zero."""
    box = syn.Box((4, 2, 1), 1)
    state = syn.gas_state(np.random.default_rng(5), box)
    buf = box.empty(0.0)
    sv, bv = box.valid(state), box.valid(buf)
    cells = [((1.0, 1.0, 0.0, 0.0, 1.0), (1.0, 0.0, 1.0, 0.0, 0.1)),
             ((1.0, 1.0, 0.0, 0.0, 1.0), (1.0, 1.0, 0.0, 0.0, 0.1)),
             ((1.0, 1.0, 0.0, 0.0, 1.0), (1.0, -0.3, 0.0, 0.0, 0.1)),
             ((1.3, 0.2, 0.0, 0.0, 0.8), (0.2, 3.0, -4.0, 1.5, 0.9)),
             (None, (0.1, 0.0, 0.0, 0.0, 0.2))]
    for c, (U, D) in enumerate(cells):
        if U is not None:
            sv[:, 0, c // 4, c % 4] = U
        bv[:, 0, c // 4, c % 4] = D
    return box, state, buf


def test_feedback_apply_without_a_feasible_lambda(orc):
    """Steps 3 + 5 alone on cells where Eq. lambda has no feasible value (the
    reading: lambda = 0, counted), beside a limited cell and a change without
    momentum: state, eta and both counters bit for bit against the oracle."""
    import torch

    from paper_2509_18261_gb300 import pmp

    box, state, buf = lambda_case_cells()
    params = syn.feedback_params()
    want = state.copy()
    eta_want, counts_want = orc.apply(params, box, want, buf.copy(), want_eta=True)
    assert counts_want[1] == 3 and counts_want[0] == 4
    ctx = pmp.Context(params)
    try:
        st = pmp.Mesh(torch.from_numpy(state.copy()).to("cuda"), box.n, box.g)
        bm = pmp.Mesh(torch.from_numpy(buf.copy()).to("cuda"), box.n, box.g)
        eta = torch.empty(box.ncells_valid, dtype=torch.float64, device="cuda")
        pmp.pmp_apply_limited(ctx, st, bm, eta_out=eta)
        counts = pmp.pmp_limiter_counts(ctx)
        assert pmp.pmp_get_error(ctx) == (0, -1)
    finally:
        ctx.close()
    assert_bits_equal(valid_flat(box, st.data.cpu().numpy()), valid_flat(box, want), "state after Step 5")
    assert_bits_equal(eta.cpu().numpy(), eta_want, "eta")
    assert tuple(counts) == (counts_want[0], counts_want[1])


@pytest.mark.parametrize("kind", ["feedback", "sink"])
def test_no_particles(orc, kind):
    box = syn.Box((6, 6, 6), 4)
    state = syn.gas_state(np.random.default_rng(1), box)
    empty = {k: np.zeros(0) for k in ("x", "y", "z", "m", "px", "py", "pz", "e")}
    params = syn.feedback_params() if kind == "feedback" else syn.sink_params()
    g = gpu_pass(params, box, state, empty)
    assert_bits_equal(valid_flat(box, g["state"]), valid_flat(box, state), "state unchanged")
    assert np.all(box.grid(g["buf"]) == 0.0)


def test_sorted_mode_is_reproducible(orc):
    w = syn.make_workload("c1_32")
    a = gpu_pass(w["fb_params"], w["box"], w["state"], w["fb"], mode="sorted")
    b = gpu_pass(w["fb_params"], w["box"], w["state"], w["fb"], mode="sorted")
    assert_bits_equal(a["state"], b["state"], "two sorted runs")


@pytest.mark.parametrize("mode", ["sorted", "atomic"])
@pytest.mark.parametrize(
    "n,g,rK,S,periodic",
    [((12, 10, 9), 4, 2.0, 4, (1, 1, 1)), ((7, 8, 6), 3, 2.5, 3, (1, 0, 1)), ((5, 5, 5), 2, 1.0, 1, (0, 0, 0))],
)
def test_mass_deposit(orc, mode, n, g, rK, S, periodic):
    """Particle-mesh kind (Steps 1, 2, 5): every row spread by omega."""
    rng = np.random.default_rng(31 + g)
    box = syn.Box(n, g)
    state = syn.gas_state(rng, box)
    parts = _cloud(rng, n, 40)
    g_, ref = _check_pass(orc, syn.mass_params(r_K=rK, subsample=S), box, state, parts, mode, periodic=periodic)
    assert ref["counts"][0] == 0
    for k in parts:
        assert_bits_equal(g_["parts"][k], parts[k], f"particle {k} unchanged")


def test_mass_deposit_without_energy(orc):
    rng = np.random.default_rng(5)
    box = syn.Box((10, 10, 10), 4)
    state = syn.gas_state(rng, box)
    parts = _cloud(rng, box.n, 20)
    no_e = {k: v for k, v in parts.items() if k != "e"}
    g = gpu_pass(syn.mass_params(), box, state, no_e, mode="sorted")
    zero_e = dict(parts, e=np.zeros(20))
    ref = oracle_pass(orc, syn.mass_params(), box, state, zero_e)
    assert_bits_equal(valid_flat(box, g["state"]), valid_flat(box, ref["state"]), "state")
    assert np.all(box.valid(g["buf"])[4] == 0.0)


@pytest.mark.parametrize("kind", ["feedback", "sink"])
def test_sorted_mode_long_runs(orc, kind):
    """Clustered particles: many buffer cells take more contributions than a
    warp has lanes, so the sorted mode's warp-per-run path runs; still the
    oracle's bits."""
    rng = np.random.default_rng(17)
    box = syn.Box((16, 14, 12), 4)
    state = syn.gas_state(rng, box)
    parts = syn.particles(rng, box.n, 600, kind, clustered=600, nclusters=2)
    params = syn.feedback_params() if kind == "feedback" else syn.sink_params(dt=0.01)
    _, ref = _check_pass(orc, params, box, state, parts, "sorted")
    # contributions per cell: at least one cell with more than 32
    n = np.zeros(box.ncells_padded)
    for s in range(len(parts["x"])):
        one = {k: v[s:s + 1] for k, v in parts.items()}
        ijk, _ = orc.deltas(params, box, state, one)
        g = box.g
        px, py = box.padded[0], box.padded[1]
        for i, j, k in ijk:
            n[((k + g) * py + (j + g)) * px + (i + g)] += 1
    assert n.max() > 32
