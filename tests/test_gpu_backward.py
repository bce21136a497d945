"""The hand-written adjoint of a supernova pass (pmp_backward) on the GPU.

- dot-product identity <J dtheta, v> = <dtheta, J^T v> against the dual-number
  oracle (forward mode), to 1e-8 relative;
- fourth-order central finite differences of the C oracle's deposition
  function on 64 particles of the 128^3 workload whose kernels touch no
  limiter-active cell, at 1e-8 relative plus the quotient's rounding
  allowance;
- cells where the limiter acted pass no gradient;
- the autograd Function returns exactly pmp_backward's gradients.
"""
import math

import numpy as np
import pytest

from paper_2509_18261_gb300 import synthetic as syn
from helpers import fd_derivative

pytestmark = pytest.mark.gpu
FIELDS = ("m", "e", "px", "py", "pz", "x", "y", "z")


def _run(params, box, state_np, parts_np, mode, gU_np):
    import torch

    from paper_2509_18261_gb300 import pmp

    u_old = torch.from_numpy(state_np.copy()).cuda()
    u_new = u_old.clone()
    parts = pmp.parts_to_device(parts_np)
    ps = pmp.Pass(params, box, u_new, parts, mode=mode, want_eta=True)
    ps.run()
    n = len(parts_np["x"])
    g = torch.zeros((8, n), dtype=torch.float64, device="cuda")
    gU = torch.from_numpy(gU_np).cuda()
    pmp.pmp_backward(ps.ctx, pmp.Mesh(u_old, box.n, box.g), ps.buffer, parts, ps.gathered_view(), gU, g,
                     ps.workspace)
    torch.cuda.synchronize()
    out = g.cpu().numpy(), ps.eta.cpu().numpy(), pmp.pmp_get_error(ps.ctx)
    ps.ctx.close()
    return out


def test_adjoint_dot_product_identity(orc):
    from oracle import dual

    rng = np.random.default_rng(31)
    box = syn.Box((16, 16, 16), 2)
    state = syn.gas_state(rng, box)
    parts = syn.particles(rng, box.n, 24, "feedback", clustered=8, nclusters=2)
    params = syn.feedback_params()
    v = box.empty(0.0)
    box.valid(v)[...] = rng.standard_normal((5,) + box.n[::-1])
    g, eta, err = _run(params, box, state, parts, "sorted", v)
    assert err == (0, -1)
    ref = orc.cycle(params, box, state.copy(), {k: a.copy() for k, a in parts.items()}, want_eta=True)
    assert np.array_equal(eta, ref["eta"]), "limiter decisions"
    passmask = (ref["eta"] == 1.0).reshape(box.n[::-1])
    assert not passmask.all(), "the case should exercise limiter-active cells"
    dth = {k: rng.standard_normal(len(parts["x"])) for k in FIELDS}
    for k in ("x", "y", "z"):
        dth[k] *= 1e-2
    _, tan = dual.pass_tangent(orc, params, box, state, parts, dth, passmask)
    lhs = math.fsum((box.valid(v) * tan).ravel())
    rhs = math.fsum(float(dth[k][s] * g[i, s]) for i, k in enumerate(FIELDS) for s in range(len(parts["x"])))
    scale = math.fsum(abs(float(dth[k][s] * g[i, s])) for i, k in enumerate(FIELDS) for s in range(len(parts["x"])))
    assert abs(lhs - rhs) <= 1e-8 * scale


def test_adjoint_matches_finite_differences_128(orc):
    """64 particles of the 128^3 workload whose kernels touch no
    limiter-active cell: each of the 8 gradients within 1e-8 of the
    fourth-order central difference of the oracle's deposition function,
    plus the difference quotient's own rounding allowance (helpers.fd_derivative)."""
    w = syn.make_workload("c4_128")
    box, state, parts, params = w["box"], w["state"], w["fb"], w["fb_params"]
    rng = np.random.default_rng(41)
    R = box.empty(0.0)
    box.valid(R)[...] = rng.standard_normal((5,) + box.n[::-1])
    g, eta, err = _run(params, box, state, parts, "atomic", R)
    assert err == (0, -1)
    nx, ny, nz = box.n
    active = (eta < 1.0).reshape(nz, ny, nx)
    Rv = box.valid(R)
    G = orc.gather(params, box, state, parts)
    order = rng.permutation(len(parts["x"]))
    checked = decided = total = 0
    for s in order:
        if checked >= 64:
            break
        one = {k: parts[k][s:s + 1].copy() for k in FIELDS}
        ijk, _ = orc.kernel_of(params, box, one["x"][0], one["y"][0], one["z"][0])
        if any(active[k % nz, j % ny, i % nx] for (i, j, k) in ijk):
            continue
        for i, f in enumerate(FIELDS):
            r = fd_derivative(orc, params, box, state, one, Rv, f, G[0, s])
            if r is None:
                continue
            fd, floor = r
            total += 1
            decided += floor <= 1e-9 * abs(fd)
            gi = g[i, s]
            assert abs(gi - fd) <= 1e-8 * abs(fd) + floor, (
                f"particle {s} d/d{f}: adjoint {gi!r} vs finite difference {fd!r} "
                f"(rel {abs(gi - fd) / abs(fd):.2e}, floor {floor / abs(fd):.2e})")
        checked += 1
    assert checked == 64
    assert total >= 64 * 7
    assert decided >= total // 2  # most checks are settled by the 1e-8 term, not the floor


def test_limiter_active_cells_pass_no_gradient(orc):
    rng = np.random.default_rng(51)
    box = syn.Box((16, 16, 16), 2)
    state = syn.gas_state(rng, box)
    parts = syn.particles(rng, box.n, 40, "feedback")
    params = syn.feedback_params()
    probe = box.empty(0.0)
    _, eta, _ = _run(params, box, state, parts, "atomic", probe)
    active = (eta < 1.0).reshape(box.n[::-1])
    assert active.any()
    gU = box.empty(0.0)
    box.valid(gU)[:, active] = rng.standard_normal((5, int(active.sum())))
    g, _, _ = _run(params, box, state, parts, "atomic", gU)
    assert np.all(g == 0.0)


def test_autograd_function_matches_c_abi():
    import torch

    from paper_2509_18261_gb300 import pmp
    from paper_2509_18261_gb300.autograd import feedback_pass

    rng = np.random.default_rng(61)
    box = syn.Box((16, 16, 16), 2)
    state = syn.gas_state(rng, box)
    parts_np = syn.particles(rng, box.n, 30, "feedback")
    params = syn.feedback_params()
    R = box.empty(0.0)
    box.valid(R)[...] = rng.standard_normal((5,) + box.n[::-1])
    leaves = {k: torch.from_numpy(v.copy()).cuda().requires_grad_(True) for k, v in parts_np.items()}
    u = torch.from_numpy(state).cuda()
    u_new = feedback_pass(u, leaves, params, box)
    Rt = torch.from_numpy(R).cuda()
    loss = (torch.nan_to_num(u_new) * Rt).sum()
    loss.backward()
    g, _, _ = _run(params, box, state, parts_np, "atomic", R)
    for i, k in enumerate(FIELDS):
        assert np.array_equal(leaves[k].grad.cpu().numpy(), g[i]), k
