"""Sink creation (Sec. 3.1.2) on the GPU through the C ABI, against the oracle:
the number of qualifying cells, the new sinks (position, mass, momentum, in
cell order) and the updated state bit for bit; a capacity smaller than the
number of qualifying cells; creation after a real accretion pass."""
import numpy as np
import pytest

from paper_2509_18261_gb300 import synthetic as syn
from helpers import assert_bits_equal, valid_flat

pytestmark = pytest.mark.gpu

KEYS = ("x", "y", "z", "m", "px", "py", "pz")


def _gpu_create(params, box, state, buf, cap, periodic=(1, 1, 1)):
    import torch

    from paper_2509_18261_gb300 import pmp

    st = torch.from_numpy(state.copy()).cuda()
    b = torch.from_numpy(buf.copy()).cuda()
    ctx = pmp.Context(params)
    S = pmp.Mesh(st, box.n, box.g, periodic)
    B = pmp.Mesh(b, box.n, box.g, periodic)
    ws = torch.empty(pmp.pmp_create_sinks_workspace_size(ctx, S), dtype=torch.uint8, device="cuda")
    out = {k: torch.full((max(cap, 1),), -1.0, dtype=torch.float64, device="cuda") for k in KEYS}
    if cap == 0:
        out = {k: v[:0] for k, v in out.items()}
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    pmp.pmp_create_sinks(ctx, S, B, out, cnt, ws)
    torch.cuda.synchronize()
    err = pmp.pmp_get_error(ctx)
    ctx.close()
    assert err == (0, -1)
    return int(cnt.item()), {k: v.cpu().numpy() for k, v in out.items()}, st.cpu().numpy()


def _case(seed, n=(14, 12, 10)):
    rng = np.random.default_rng(seed)
    box = syn.Box(n, 4)
    state = syn.gas_state(rng, box)
    buf = box.empty(0.0)
    bv = box.valid(buf)
    bv[:, rng.random(bv.shape[1:]) < 0.3] = -1e-3
    return box, state, buf


@pytest.mark.parametrize("periodic", [(1, 1, 1), (1, 0, 1)])
def test_create_matches_oracle(orc, periodic):
    box, state, buf = _case(3)
    params = syn.sink_params(G=0.3)
    ref_state = state.copy()
    n_ref, ref = orc.create_sinks(params, box, ref_state, buf, periodic=periodic)
    assert n_ref > 3
    n, got, st = _gpu_create(params, box, state, buf, box.ncells_valid, periodic)
    assert n == n_ref
    for k in KEYS:
        assert_bits_equal(got[k][:n], ref[k], f"new sink {k}")
    assert_bits_equal(valid_flat(box, st), valid_flat(box, ref_state), "state after creation")


def test_capacity_limits_creation(orc):
    box, state, buf = _case(3)
    params = syn.sink_params(G=0.3)
    ref_state = state.copy()
    n_ref, ref = orc.create_sinks(params, box, ref_state, buf, cap=3)
    assert n_ref > 3
    n, got, st = _gpu_create(params, box, state, buf, 3)
    assert n == n_ref
    for k in KEYS:
        assert_bits_equal(got[k], ref[k], f"new sink {k}")
    assert_bits_equal(valid_flat(box, st), valid_flat(box, ref_state), "state: only the first 3 cells change")


def test_create_after_accretion_pass(orc):
    """The 32^3 workload's sink pass (sorted deposit), its summed buffer kept,
    then creation; denser gas so that some cells exceed rho_Tr."""
    import torch

    from paper_2509_18261_gb300 import pmp

    w = syn.make_workload("c1_32")
    box = w["box"]
    state = w["state"].copy()
    box.valid(state)[:] *= 4.0
    params = syn.sink_params(G=0.1)
    ref_state = state.copy()
    ref_parts = {k: v.copy() for k, v in w["sink"].items()}
    r = orc.cycle(params, box, ref_state, ref_parts)
    n_ref, ref = orc.create_sinks(params, box, ref_state, r["buf"])
    st = torch.from_numpy(state.copy()).cuda()
    ps = pmp.Pass(params, box, st, pmp.parts_to_device(w["sink"]), mode="sorted")
    ps.run()
    ws = torch.empty(pmp.pmp_create_sinks_workspace_size(ps.ctx, ps.state), dtype=torch.uint8, device="cuda")
    out = {k: torch.zeros(box.ncells_valid, dtype=torch.float64, device="cuda") for k in KEYS}
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    pmp.pmp_create_sinks(ps.ctx, ps.state, ps.buffer, out, cnt, ws)
    torch.cuda.synchronize()
    assert pmp.pmp_get_error(ps.ctx) == (0, -1)
    n = int(cnt.item())
    assert n == n_ref and n > 0
    for k in KEYS:
        assert_bits_equal(out[k][:n].cpu().numpy(), ref[k], f"new sink {k}")
    assert_bits_equal(valid_flat(box, st.cpu().numpy()), valid_flat(box, ref_state), "state")
    ps.ctx.close()


def test_create_rejects_wrong_kind_and_missing_arrays():
    import torch

    from paper_2509_18261_gb300 import pmp

    box, state, buf = _case(5)
    st = torch.from_numpy(state).cuda()
    b = torch.from_numpy(buf).cuda()
    S, B = pmp.Mesh(st, box.n, box.g), pmp.Mesh(b, box.n, box.g)
    fb = pmp.Context(syn.feedback_params())
    with pytest.raises(pmp.PMPError):
        pmp.pmp_create_sinks_workspace_size(fb, S)
    fb.close()
    sk = pmp.Context(syn.sink_params())
    ws = torch.empty(pmp.pmp_create_sinks_workspace_size(sk, S), dtype=torch.uint8, device="cuda")
    out = {k: torch.zeros(4, dtype=torch.float64, device="cuda") for k in KEYS}
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(pmp.PMPError):
        pmp.pmp_create_sinks(sk, S, B, out, cnt, ws[: ws.numel() // 2])
    sk.close()


def test_auxiliary_fields_under_accretion(orc):
    """pmp_apply_extra between Step 2 and Step 5 of a sink pass: the extra
    fields, the state and the sinks equal the oracle's bit for bit."""
    import torch

    from paper_2509_18261_gb300 import pmp

    rng = np.random.default_rng(12)
    box = syn.Box((14, 12, 10), 4)
    state = syn.gas_state(rng, box)
    box.valid(state)[:] *= 3.0
    parts = syn.particles(rng, box.n, 12, "sink")
    params = syn.sink_params(dt=1.0)
    X = np.zeros((3, box.field_stride))
    X[0] = state[0] * rng.uniform(0.0, 1.0, box.field_stride)
    X[1] = state[0] * 1.5
    X[2] = state[0]
    X = np.nan_to_num(X)
    # oracle: gather, deposit, fold, extra, Step 4, Step 5
    st_r, p_r, X_r = state.copy(), {k: v.copy() for k, v in parts.items()}, X.copy()
    G = orc.gather(params, box, st_r, p_r)
    buf = box.empty(0.0)
    orc.deposit(params, box, st_r, p_r, G, buf)
    orc.fold(box, buf)
    orc.apply_extra(params, box, st_r, buf, X_r)
    orc.return_sinks(params, box, st_r, buf, p_r, G)
    orc.apply(params, box, st_r, buf)
    # GPU, sorted deposit
    st = torch.from_numpy(state.copy()).cuda()
    pd = pmp.parts_to_device(parts)
    Xd = torch.from_numpy(X.copy()).cuda()
    ps = pmp.Pass(params, box, st, pd, mode="sorted")
    c = ps.ctx
    pmp.pmp_zero_buffer(c, ps.buffer)
    pmp.pmp_gather(c, ps.state, pd, ps.gathered, "sorted", ps.workspace)
    pmp.pmp_deposit(c, ps.state, pd, ps.gathered, ps.buffer, "sorted", ps.workspace)
    pmp.pmp_fold_ghosts(c, ps.buffer)
    pmp.pmp_apply_extra(c, ps.state, ps.buffer, Xd)
    pmp.pmp_apply_limited(c, ps.state, ps.buffer, pd, ps.gathered, None, ps.workspace)
    torch.cuda.synchronize()
    assert pmp.pmp_get_error(c) == (0, -1)
    got = Xd.cpu().numpy()
    for f in range(3):
        assert_bits_equal(box.valid(got[f:f + 1])[0], box.valid(X_r[f:f + 1])[0], f"extra field {f}")
    assert_bits_equal(valid_flat(box, st.cpu().numpy()), valid_flat(box, st_r), "state")
    for k in ("m", "px", "py", "pz"):
        assert_bits_equal(pd[k].cpu().numpy(), p_r[k], f"sink {k}")
    c.close()
