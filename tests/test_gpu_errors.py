"""Error behaviour of the C ABI on a GPU: host-side argument errors raise and
enqueue nothing; device-side input errors set the status word (first code and
index) without trapping."""
import math

import numpy as np
import pytest

from paper_2509_18261_gb300 import synthetic as syn
from helpers import gpu_pass

pytestmark = pytest.mark.gpu


def _cloud(n, count, seed=3):
    rng = np.random.default_rng(seed)
    x = [rng.uniform(0, n[a], count) for a in range(3)]
    m = np.full(count, 0.01)
    return dict(x=x[0], y=x[1], z=x[2], m=m, px=m * 0.1, py=m * 0.0, pz=m * -0.1, e=np.ones(count))


@pytest.mark.parametrize("kind", ["feedback", "sink"])
def test_particle_outside_is_reported_with_its_index(kind):
    box = syn.Box((8, 8, 8), 4)
    state = syn.gas_state(np.random.default_rng(1), box)
    p = _cloud(box.n, 6)
    p["x"][3] = 8.0  # x == n is outside [0, n)
    params = syn.feedback_params() if kind == "feedback" else syn.sink_params()
    g = gpu_pass(params, box, state, p)
    assert g["error"] == (3, 3)
    assert np.all(np.isfinite(box.valid(g["state"])))


def test_nan_position_is_reported():
    box = syn.Box((8, 8, 8), 2)
    state = syn.gas_state(np.random.default_rng(1), box)
    p = _cloud(box.n, 5)
    p["z"][2] = math.nan
    g = gpu_pass(syn.feedback_params(), box, state, p)
    assert g["error"] == (4, 2)


def test_nonpositive_mass_is_reported():
    box = syn.Box((8, 8, 8), 2)
    state = syn.gas_state(np.random.default_rng(1), box)
    p = _cloud(box.n, 5)
    p["m"][1] = 0.0
    g = gpu_pass(syn.feedback_params(), box, state, p)
    assert g["error"][0] == 4 and g["error"][1] == 1


def test_host_argument_errors_raise():
    import torch

    from paper_2509_18261_gb300 import pmp

    with pytest.raises(pmp.PMPError) as e:
        pmp.Context(syn.feedback_params(r_K=0.5))
    assert e.value.code == 1
    box = syn.Box((8, 8, 8), 1)  # ghost width 1 < ceil(r_K) = 2
    st = torch.from_numpy(syn.gas_state(np.random.default_rng(1), box)).cuda()
    parts = pmp.parts_to_device(_cloud(box.n, 4))
    ps = pmp.Pass(syn.feedback_params(), box, st, parts)
    pmp.pmp_gather(ps.ctx, ps.state, parts, ps.gathered, "atomic", ps.workspace)
    with pytest.raises(pmp.PMPError) as e:
        pmp.pmp_deposit(ps.ctx, ps.state, parts, ps.gathered, ps.buffer, "atomic", ps.workspace)
    assert e.value.code == 2
    box2 = syn.Box((8, 8, 8), 2)
    st2 = torch.from_numpy(syn.gas_state(np.random.default_rng(1), box2)).cuda()
    ps2 = pmp.Pass(syn.feedback_params(), box2, st2, parts, mode="sorted")
    with pytest.raises(pmp.PMPError) as e:  # workspace smaller than pmp_workspace_size
        pmp.pmp_gather(ps2.ctx, ps2.state, parts, ps2.gathered, "sorted", ps2.workspace[:1024])
    assert e.value.code == 6
    pmp.pmp_gather(ps2.ctx, ps2.state, parts, ps2.gathered, "sorted", ps2.workspace)
    with pytest.raises(pmp.PMPError) as e:  # a plan built for another mode
        pmp.pmp_deposit(ps2.ctx, ps2.state, parts, ps2.gathered, ps2.buffer, "atomic", ps2.workspace)
    assert e.value.code == 6
    with pytest.raises(pmp.PMPError) as e:  # state and buffer may not overlap
        pmp.pmp_deposit(ps2.ctx, ps2.state, parts, ps2.gathered, ps2.state, "sorted", ps2.workspace)
    assert e.value.code == 1
    assert pmp.pmp_get_error(ps2.ctx) == (0, -1)


def test_new_entry_points_check_their_arguments():
    """The rounded mode's workspace, pmp_apply_extra and the batched form's
    kinds: host-side errors raise and enqueue nothing."""
    import torch

    from paper_2509_18261_gb300 import pmp

    box = syn.Box((8, 8, 8), 4)
    st = torch.from_numpy(syn.gas_state(np.random.default_rng(1), box)).cuda()
    parts = pmp.parts_to_device(_cloud(box.n, 4))
    # ROUNDED needs the error-bound part of the workspace (sized from the buffer)
    ps = pmp.Pass(syn.feedback_params(), box, st, parts, mode="rounded")
    n_atomic = pmp.pmp_workspace_size(ps.ctx, ps.buffer, 4, "atomic")
    assert ps.workspace.numel() >= n_atomic + 5 * box.field_stride * 8
    pmp.pmp_gather(ps.ctx, ps.state, parts, ps.gathered, "rounded", ps.workspace)
    with pytest.raises(pmp.PMPError) as e:
        pmp.pmp_deposit(ps.ctx, ps.state, parts, ps.gathered, ps.buffer, "rounded", ps.workspace[:n_atomic])
    assert e.value.code == 6
    # pmp_apply_extra: sink contexts only, and a stride covering the padded box
    extra = torch.zeros((2, box.field_stride), dtype=torch.float64, device="cuda")
    with pytest.raises(pmp.PMPError) as e:
        pmp.pmp_apply_extra(ps.ctx, ps.state, ps.buffer, extra)
    assert e.value.code == 1
    sk = pmp.Pass(syn.sink_params(), box, st, parts)
    with pytest.raises(pmp.PMPError) as e:
        pmp.pmp_apply_extra(sk.ctx, sk.state, sk.buffer, extra[:, : box.ncells_padded // 2].contiguous())
    assert e.value.code == 1
    # the batched form covers supernovae and sinks, not the particle-mesh kind
    w = syn.make_batch_workload(supergrid=(2, 2, 2), edges=(16,), xmax=50.0, seed=3)
    b = w["batch"]
    ctx = pmp.Context(syn.mass_params())
    with pytest.raises(pmp.PMPError) as e:
        pmp.BatchHandle(ctx, b.dims, b.nb, b.offset, b.fstride, b.g, b.arena_len)
    assert e.value.code == 1
    ctx.close()
    assert pmp.pmp_get_error(ps.ctx) == (0, -1)
    ps.ctx.close()
    sk.ctx.close()
