"""Cells of size dx != 1 on the GPU, against the oracle, through the C ABI.

The cell size enters the path in a few places only: V = dx^3 in the gathered
volumes and masses, in Step 4 and in the conservation of every deposit;
rho_Tr = J^2 pi c_s^2 / (G dx^2) (Eq. truelove); and r_acc = r_BH / dx
(Sec. 3.1.1).  The sorted mode stays bit-exact against the oracle at
dx = 0.5 for both kinds, and the atomic mode within its tolerance.
"""
import math

import numpy as np
import pytest

from paper_2509_18261_gb300 import synthetic as syn
from helpers import assert_bits_equal, assert_state_within_bound, gpu_pass, oracle_pass, sink_return_bound, valid_flat

pytestmark = pytest.mark.gpu


def _cloud(rng, n, count):
    x = rng.uniform(0, n[0], count)
    y = rng.uniform(0, n[1], count)
    z = rng.uniform(0, n[2], count)
    m = np.exp(rng.uniform(math.log(1e-3), math.log(1e-1), count))
    v = rng.normal(0, 0.1, (3, count))
    return dict(x=x, y=y, z=z, m=m, px=m * v[0], py=m * v[1], pz=m * v[2], e=np.ones(count))


@pytest.mark.parametrize("mode", ["sorted", "atomic"])
@pytest.mark.parametrize("kind", ["feedback", "sink"])
def test_half_cell_size(orc, kind, mode):
    dx = 0.5
    rng = np.random.default_rng(41 if kind == "feedback" else 43)
    n = (10, 9, 11)
    box = syn.Box(n, 4)
    state = syn.gas_state(rng, box)
    parts = _cloud(rng, n, 16)
    if kind == "feedback":
        params = syn.feedback_params()
    else:
        v = box.valid(state)
        v[0] *= 20.0  # dense enough for the Truelove branch at dx = 0.5
        v[4] *= 20.0
        parts["m"] = np.exp(rng.uniform(0, math.log(100), 16))
        params = syn.sink_params(dt=0.5)
    ref = oracle_pass(orc, params, box, state, parts, dx=dx)
    g = gpu_pass(params, box, state, parts, mode=mode, dx=dx)
    assert g["error"] == (0, -1), g["error"]
    assert_bits_equal(g["gathered"], ref["gathered"], "gathered rows")
    if mode == "sorted":
        assert_bits_equal(valid_flat(box, g["state"]), valid_flat(box, ref["state"]), "state after Step 5")
        assert_bits_equal(g["eta"], ref["eta"], "eta")
        if kind == "sink":
            for k in ("m", "px", "py", "pz"):
                assert_bits_equal(g["parts"][k], ref["parts"][k], f"sink {k} after Step 4")
    else:
        A = valid_flat(box, ref["absbuf"])
        assert_state_within_bound(params, valid_flat(box, state), valid_flat(box, ref["buf"]), A, ref["eta"],
                                  valid_flat(box, g["state"]), valid_flat(box, ref["state"]))
        if kind == "sink":
            for k in ("m", "px", "py", "pz"):
                tol = sink_return_bound(params, box, state, parts, ref["parts"], k)
                assert np.all(np.abs(g["parts"][k] - ref["parts"][k]) <= tol), k
    if kind == "sink":
        assert ref["counts"][0] > 0
