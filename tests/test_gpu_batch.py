"""The batched form on the GPU (pmp_cycle_batched) against the oracle's
batched pass, through the C ABI.

- the deterministic strategies (OWNER_CUBE, OWNER_ROWS) give the oracle's
  bits: gathered rows, the whole buffer arena (ghost deposits and folded
  sums), the state arena (ghost cells untouched), eta, sink masses and
  momenta, limiter counts -- for the persistent launch, its CUDA graph and
  the per-patch launch loop;
- the atomic strategy agrees within 1e-12 of sum |dU| per cell and field;
- the autotuner's choice (deterministic) still gives the oracle's bits;
- the uneven 512-patch workload (8x8x8 super-grid, edges 16..64, power-law
  counts): the mixed cycle, supernovae then sinks, bit-exact;
- argument checks of pmp_batch_create / pmp_batch_set_particles;
- a grid barrier held on purpose (pmp_batch_hold_barriers): the bounded wait
  ends the pass with PMP_ERR_TIMEOUT, and the context stays usable.
"""
import numpy as np
import pytest

from paper_2509_18261_gb300 import synthetic as syn
from helpers import assert_bits_equal, assert_within_abs

pytestmark = pytest.mark.gpu


def _small(kind, seed=7):
    w = syn.make_batch_workload(supergrid=(3, 2, 2), edges=(16, 24), xmax=2000.0, seed=seed)
    if kind == "feedback":
        return w["batch"], w["state"], w["fb"], w["fb_first"], w["fb_params"]
    return w["batch"], w["state"], w["sink"], w["sink_first"], syn.sink_params(dt=2.0)


def _gpu(params, batch, state_np, parts_np, first, launch="persistent", strategy=None, autotune=None):
    import torch

    from paper_2509_18261_gb300 import pmp

    st = torch.from_numpy(state_np.copy()).cuda()
    parts = pmp.parts_to_device(parts_np)
    bp = pmp.BatchPass(params, batch, st, parts, first, want_eta=True)
    chosen = None
    if strategy is not None:
        pmp.pmp_batch_set_strategy(bp.h, strategy)
    if autotune is not None:
        chosen = pmp.pmp_batch_autotune(bp.h, st, bp.buffer, parts, bp.gathered, deterministic=autotune)
    bp.run(launch)
    torch.cuda.synchronize()
    out = dict(state=st.cpu().numpy(), buf=bp.buffer.cpu().numpy(), eta=bp.eta.cpu().numpy(),
               gathered=bp.gathered_view().cpu().numpy(), parts={k: v.cpu().numpy() for k, v in parts.items()},
               error=pmp.pmp_get_error(bp.ctx), counts=pmp.pmp_limiter_counts(bp.ctx), chosen=chosen,
               strategies=pmp.pmp_batch_strategies(bp.h))
    bp.close()
    return out


def _oracle(orc, params, batch, state_np, parts_np, first):
    st = state_np.copy()
    parts = {k: v.copy() for k, v in parts_np.items()}
    r = orc.batch_cycle(params, batch, st, parts, first, want_abs=True, want_eta=True)
    r["state"], r["parts"] = st, parts
    return r


def _assert_same(got, ref, kind, what):
    assert got["error"] == (0, -1), what
    assert_bits_equal(got["gathered"], ref["gathered"], f"{what}: gathered")
    assert_bits_equal(got["buf"], ref["buf"], f"{what}: buffer arena")
    assert_bits_equal(got["state"], ref["state"], f"{what}: state arena")
    assert_bits_equal(got["eta"], ref["eta"], f"{what}: eta")
    if kind == "sink":
        for k in ("m", "px", "py", "pz"):
            assert_bits_equal(got["parts"][k], ref["parts"][k], f"{what}: sink {k}")
    assert tuple(got["counts"]) == tuple(int(v) for v in ref["counts"]), what


@pytest.mark.parametrize("kind", ["feedback", "sink"])
@pytest.mark.parametrize("launch", ["persistent", "per_patch", "graph"])
def test_batch_deterministic_is_bit_exact(orc, kind, launch):
    batch, state, parts, first, params = _small(kind)
    assert first[-1] > 10
    ref = _oracle(orc, params, batch, state, parts, first)
    got = _gpu(params, batch, state, parts, first, launch=launch)
    _assert_same(got, ref, kind, f"{kind}/{launch}")
    if kind == "sink":
        assert ref["counts"][0] > 0


@pytest.mark.parametrize("kind", ["feedback", "sink"])
def test_owner_rows_strategy_is_bit_exact(orc, kind):
    batch, state, parts, first, params = _small(kind, seed=13)
    ref = _oracle(orc, params, batch, state, parts, first)
    got = _gpu(params, batch, state, parts, first, strategy="owner_rows")
    assert set(got["strategies"]) == {1}
    _assert_same(got, ref, kind, f"{kind}/owner_rows")


@pytest.mark.parametrize("kind", ["feedback", "sink"])
def test_atomic_strategy_within_tolerance(orc, kind):
    batch, state, parts, first, params = _small(kind, seed=13)
    ref = _oracle(orc, params, batch, state, parts, first)
    got = _gpu(params, batch, state, parts, first, strategy="atomic")
    assert got["error"] == (0, -1)
    assert_bits_equal(got["gathered"], ref["gathered"], "gathered")
    A = ref["absbuf"]
    assert_within_abs(got["buf"], ref["buf"], A, "buffer arena")
    same = (got["eta"] == 1.0) & (ref["eta"] == 1.0)
    for p in range(batch.np):
        lo, hi = batch.vbase[p], batch.vbase[p + 1]
        m = same[lo:hi].reshape(batch.valid(ref["state"], p).shape[1:])
        g, r, a = batch.valid(got["state"], p), batch.valid(ref["state"], p), batch.valid(A, p)
        assert np.all(np.abs(g - r)[:, m] <= 1e-12 * (np.abs(r) + a)[:, m]), f"patch {p}"
    assert np.all(np.abs(got["eta"] - ref["eta"]) <= 1e-9)


def test_autotuned_deterministic_choice_is_bit_exact(orc):
    batch, state, parts, first, params = _small("feedback", seed=13)
    ref = _oracle(orc, params, batch, state, parts, first)
    got = _gpu(params, batch, state, parts, first, autotune=True)
    assert all(c in (-1, 0, 1) for c in got["chosen"])
    assert any(c >= 0 for c in got["chosen"])
    _assert_same(got, ref, "feedback", "autotuned")


def test_particle_outside_its_patch_is_reported(orc):
    batch, state, parts, first, params = _small("feedback")
    bad = {k: v.copy() for k, v in parts.items()}
    s = int(first[1])  # first particle of patch 1
    bad["x"][s] = float(batch.dims[1][0]) + 0.5
    got = _gpu(params, batch, state, bad, first)
    assert got["error"] == (3, s)
    assert np.all(got["gathered"][:, s] == 0.0)


def test_batch_create_rejects_bad_tables():
    import torch

    from paper_2509_18261_gb300 import pmp

    batch, _, _, _, params = _small("feedback")
    ctx = pmp.Context(params)
    dims, nb = batch.dims.copy(), batch.nb.copy()
    off, fs = batch.offset.copy(), batch.fstride.copy()

    def code(**kw):
        a = dict(dims=dims, nb=nb, offset=off, field_stride=fs, ng=4, arena_len=batch.arena_len)
        a.update(kw)
        with pytest.raises(pmp.PMPError) as e:
            pmp.BatchHandle(ctx, a["dims"], a["nb"], a["offset"], a["field_stride"], a["ng"], a["arena_len"])
        return e.value.code

    assert code(ng=1) == 2  # ghost thinner than ceil(r_K)
    nb2 = nb.copy()
    assert syn.NB_OFFSETS[13] == (1, 0, 0) and nb[0, 13] == 1
    nb2[0, 13] = 2  # +x neighbour of patch 0 said to be patch 2: not reciprocal
    assert code(nb=nb2) == 1
    dims2 = dims.copy()
    dims2[1, 1] = 24 if dims2[1, 1] == 16 else 16  # extent across +x does not match
    assert code(dims=dims2) == 1
    off2 = off.copy()
    off2[1] = off2[0] + 8  # overlapping patches
    assert code(offset=off2) == 1
    assert code(arena_len=batch.arena_len - 1) == 1
    h = pmp.BatchHandle(ctx, dims, nb, off, fs, 4, batch.arena_len)
    with pytest.raises(pmp.PMPError):
        pmp.pmp_batch_set_particles(h, [0] + [5] * (batch.np - 1) + [4])  # decreasing
    h.close()
    ctx.close()
    torch.cuda.synchronize()


def test_c3_uneven_512_patches_mixed_cycle_bit_exact(orc):
    w = syn.make_batch_workload()
    batch = w["batch"]
    assert batch.np == 512
    st_ref = w["state"].copy()
    fb_ref = orc.batch_cycle(w["fb_params"], batch, st_ref, {k: v.copy() for k, v in w["fb"].items()},
                             w["fb_first"], want_eta=True)
    sk_parts = {k: v.copy() for k, v in w["sink"].items()}
    sk_ref = orc.batch_cycle(w["sink_params"], batch, st_ref, sk_parts, w["sink_first"], want_eta=True)
    assert fb_ref["counts"][0] > 0 and sk_ref["counts"][0] > 0

    import torch

    from paper_2509_18261_gb300 import pmp

    st = torch.from_numpy(w["state"].copy()).cuda()
    pf = pmp.parts_to_device(w["fb"])
    ps = pmp.parts_to_device(w["sink"])
    fb = pmp.BatchPass(w["fb_params"], batch, st, pf, w["fb_first"], want_eta=True)
    sk = pmp.BatchPass(w["sink_params"], batch, st, ps, w["sink_first"], want_eta=True)
    sk.buffer = fb.buffer  # one buffer shared by the two passes
    fb.run("graph")
    eta_fb = fb.eta.cpu().numpy()
    g_fb = fb.gathered_view().cpu().numpy()
    sk.run("graph")
    torch.cuda.synchronize()
    assert pmp.pmp_get_error(fb.ctx) == (0, -1) and pmp.pmp_get_error(sk.ctx) == (0, -1)
    assert_bits_equal(g_fb, fb_ref["gathered"], "feedback gathered")
    assert_bits_equal(eta_fb, fb_ref["eta"], "feedback eta")
    assert_bits_equal(sk.gathered_view().cpu().numpy(), sk_ref["gathered"], "sink gathered")
    assert_bits_equal(sk.eta.cpu().numpy(), sk_ref["eta"], "sink eta")
    assert_bits_equal(sk.buffer.cpu().numpy(), sk_ref["buf"], "buffer arena after the sink pass")
    assert_bits_equal(st.cpu().numpy(), st_ref, "state arena after the cycle")
    for k in ("m", "px", "py", "pz"):
        assert_bits_equal(ps[k].cpu().numpy(), sk_parts[k], f"sink {k}")
    fb.close()
    sk.close()


def test_barrier_timeout_is_reported_and_the_context_recovers(orc):
    """Failure detection without a GPU fault: pmp_batch_hold_barriers makes the
    persistent launch's grid barriers wait for one block that never arrives.
    Every wait gives up after its time limit, the pass reports
    PMP_ERR_TIMEOUT (first index -1) and returns; with the hold released, the
    next pass on the same context gives the oracle's bits."""
    import torch

    from paper_2509_18261_gb300 import pmp

    batch, state, parts_np, first, params = _small("feedback")
    ref = _oracle(orc, params, batch, state, parts_np, first)
    st = torch.from_numpy(state.copy()).cuda()
    parts = pmp.parts_to_device(parts_np)
    bp = pmp.BatchPass(params, batch, st, parts, first, want_eta=True)
    try:
        pmp.pmp_batch_hold_barriers(bp.h, 1)
        bp.run("persistent")
        assert pmp.pmp_get_error(bp.ctx) == (5, -1)  # PMP_ERR_TIMEOUT
        with pytest.raises(pmp.PMPError):
            pmp.pmp_batch_hold_barriers(bp.h, 2)
        pmp.pmp_batch_hold_barriers(bp.h, 0)
        st.copy_(torch.from_numpy(state))
        for k, v in parts_np.items():
            parts[k].copy_(torch.from_numpy(v))
        bp.run("persistent")
        torch.cuda.synchronize()
        got = dict(state=st.cpu().numpy(), buf=bp.buffer.cpu().numpy(), eta=bp.eta.cpu().numpy(),
                   gathered=bp.gathered_view().cpu().numpy(), parts={k: v.cpu().numpy() for k, v in parts.items()},
                   error=pmp.pmp_get_error(bp.ctx), counts=pmp.pmp_limiter_counts(bp.ctx))
        _assert_same(got, ref, "feedback", "after the timeout")
    finally:
        bp.close()
