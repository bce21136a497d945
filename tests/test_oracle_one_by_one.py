"""The oracle's one-by-one evaluation (Bins: or_gather_at, or_cells_at,
or_sinks_at), which gives the expected values of the full-size GPU tests,
agrees bit for bit with the oracle's whole cycle on a box small enough for
both (the 512^3 workload shrunk to 20^3 at 4x its particle density): the
gathered rows, the folded buffer, |Delta U| sums, eta and the updated state
at every valid cell, and sampled sinks after Step 4."""
import numpy as np
import pytest

from paper_2509_18261_gb300 import synthetic as syn


def _workload(kind):
    w = syn.make_workload("c5_512", n=20, count_scale=(20 / 512) ** 3 * 4)
    return w["box"], w["state"], w[kind], w[kind + "_params"]


@pytest.mark.parametrize("kind", ["fb", "sink"])
def test_one_by_one_equals_the_whole_cycle(orc, kind):
    box, state, parts, params = _workload(kind)
    assert len(parts["x"]) > 50
    st = state.copy()
    p = {k: v.copy() for k, v in parts.items()}
    r = orc.cycle(params, box, st, p, want_abs=True, want_eta=True)
    bins = orc.Bins(box, state, parts)
    # gathered rows of every particle
    G = bins.gather(params, np.arange(len(parts["x"])))
    assert np.array_equal(G.view(np.uint64), r["gathered"].view(np.uint64))
    # every valid cell
    nx, ny, nz = box.n
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ijk = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    s, a, u, e = bins.cells(params, ijk)
    buf = box.valid(r["buf"]).reshape(5, -1).T
    absb = box.valid(r["absbuf"]).reshape(5, -1).T
    new = box.valid(st).reshape(5, -1).T
    assert np.array_equal(s.view(np.uint64), buf.view(np.uint64)), "folded buffer"
    assert np.array_equal(a, absb), "|Delta U| sums"
    assert np.array_equal(u.view(np.uint64), new.view(np.uint64)), "state after Step 5"
    assert np.array_equal(e, r["eta"]), "eta"
    assert r["counts"][0] > 0
    if kind == "sink":
        sel = np.random.default_rng(3).choice(len(parts["x"]), 40, replace=False)
        want = bins.sinks(params, sel)
        for c, key in enumerate(("m", "px", "py", "pz")):
            assert np.array_equal(want[:, c].view(np.uint64), p[key][sel].view(np.uint64)), key
