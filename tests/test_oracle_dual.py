"""Pins of the dual-number oracle (oracle/dual.py) used for the adjoint tests:
its primal values equal the C oracle's summed buffer, and its tangents equal
central finite differences of the C oracle's deposition function."""
import math

import numpy as np
import pytest

from paper_2509_18261_gb300 import synthetic as syn

FIELDS = ("m", "e", "px", "py", "pz", "x", "y", "z")


def _case(seed=21, n=(12, 12, 12), count=14):
    rng = np.random.default_rng(seed)
    box = syn.Box(n, 2)
    state = syn.gas_state(rng, box)
    parts = syn.particles(rng, box.n, count, "feedback")
    return box, state, parts


def test_dual_primal_matches_c_oracle(orc):
    from oracle import dual

    box, state, parts = _case()
    params = syn.feedback_params()
    G = orc.gather(params, box, state, parts)
    buf, A = box.empty(0.0), box.empty(0.0)
    orc.deposit(params, box, state, parts, G, buf, A)
    orc.fold(box, buf, A)
    zero = {k: np.zeros_like(parts[k]) for k in FIELDS}
    val, _ = dual.pass_tangent(orc, params, box, state, parts, zero, np.ones(box.n[::-1], bool))
    assert np.all(np.abs(val - box.valid(buf)) <= 1e-13 * box.valid(A) + 1e-300)


@pytest.mark.parametrize("field", FIELDS)
def test_dual_tangent_matches_central_differences(orc, field):
    from oracle import dual

    box, state, parts = _case(seed=22, count=6)
    params = syn.feedback_params()
    rng = np.random.default_rng(5)
    R = rng.standard_normal((5,) + box.n[::-1])
    nx, ny, nz = box.n
    for s in range(len(parts["x"])):
        one = {k: parts[k][s:s + 1].copy() for k in FIELDS}
        tang = {k: np.zeros(1) for k in FIELDS}
        tang[field][0] = 1.0
        _, tan = dual.pass_tangent(orc, params, box, state, one, tang, np.ones(box.n[::-1], bool))
        want = float(np.sum(R * tan))
        h = 1e-6 * max(1.0, abs(one[field][0]))

        def L(v):
            o = {k: a.copy() for k, a in one.items()}
            o[field][0] = v
            ijk, dU = orc.deltas(params, box, state, o)
            return math.fsum(float(R[f, k % nz, j % ny, i % nx] * dU[c, f])
                             for c, (i, j, k) in enumerate(ijk) for f in range(5))

        x0 = one[field][0]
        if field in ("x", "y", "z"):
            a, b = dict(one), dict(one)
            a[field] = np.array([x0 + h]); b[field] = np.array([x0 - h])
            ka = orc.kernel_of(params, box, a["x"][0], a["y"][0], a["z"][0])
            kb = orc.kernel_of(params, box, b["x"][0], b["y"][0], b["z"][0])
            if not (np.array_equal(ka[0], kb[0]) and np.array_equal(ka[1], kb[1])):
                continue  # omega or the kernel cells change inside [x - h, x + h]
        fd = (L(x0 + h) - L(x0 - h)) / (2 * h)
        assert fd == pytest.approx(want, rel=2e-6, abs=1e-9 * (abs(want) + 1e-3))


def test_dual_tangent_vanishes_where_the_limiter_acts(orc):
    """The adjoint's definition: eta is held fixed and a cell where the
    limiter acts passes no tangent.  With every other cell marked as limited,
    the tangent is exactly zero there and unchanged elsewhere; the values do
    not depend on the mask."""
    from oracle import dual

    box, state, parts = _case(seed=23, count=4)
    params = syn.feedback_params()
    rng = np.random.default_rng(6)
    tang = {k: rng.standard_normal(len(parts["x"])) for k in FIELDS}
    full = np.ones(box.n[::-1], bool)
    k, j, i = np.indices(box.n[::-1])
    mask = (i + j + k) % 2 == 0
    val1, tan1 = dual.pass_tangent(orc, params, box, state, parts, tang, full)
    val2, tan2 = dual.pass_tangent(orc, params, box, state, parts, tang, mask)
    assert np.count_nonzero(tan1[:, ~mask]) > 20
    assert np.all(tan2[:, ~mask] == 0.0)
    assert np.array_equal(tan2[:, mask], tan1[:, mask])
    assert np.array_equal(val1, val2)


def test_fourth_order_differences_agree_with_the_dual_tangents_at_1e8(orc):
    """The finite-difference procedure of the GPU adjoint test
    (helpers.fd_derivative) against the dual-number tangents on a clustered
    box: within 1e-8 relative plus the quotient's rounding allowance, for all
    eight variables; and that allowance settles at most half the checks."""
    from oracle import dual

    from helpers import fd_derivative

    rng = np.random.default_rng(23)
    box = syn.Box((24, 24, 24), 2)
    state = syn.gas_state(rng, box)
    parts = syn.particles(rng, box.n, 16, "feedback", clustered=8, nclusters=1)
    params = syn.feedback_params()
    R = rng.standard_normal((5,) + box.n[::-1])
    G = orc.gather(params, box, state, parts)
    total = decided = 0
    for s in range(len(parts["x"])):
        one = {k: parts[k][s:s + 1].copy() for k in FIELDS}
        for f in FIELDS:
            r = fd_derivative(orc, params, box, state, one, R, f, G[0, s])
            if r is None:
                continue
            fd, floor = r
            tang = {k: np.zeros(1) for k in FIELDS}
            tang[f][0] = 1.0
            _, tan = dual.pass_tangent(orc, params, box, state, one, tang, np.ones(box.n[::-1], bool))
            want = math.fsum((R * tan).ravel())
            total += 1
            decided += floor <= 1e-9 * abs(fd)
            assert abs(fd - want) <= 1e-8 * abs(want) + floor, (s, f, fd, want, floor)
    assert total >= 16 * 7
    assert decided >= total // 2
