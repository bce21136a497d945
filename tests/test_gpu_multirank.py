"""The batched pass on several ranks on the GPU, the ranks emulated one after
the other on one device: each rank a partial batch of its local patches
(pmp_batch_create_partial), its two parts (pmp_cycle_batched_part), and the
STATE, GHOST and (sinks) FOLDED exchanges packed and unpacked by the
library's kernels (pmp_batch_pack / pmp_batch_unpack), the messages copied
between the ranks' buffers.  No kernel waits on another rank's.

Every owned patch must equal the one-rank batched pass bit for bit (OWNER
deposit strategies): state, eta, gathered rows, sink masses and momenta --
against the oracle on a small batch with particles on patch faces, edges and
corners, and against the one-rank GPU pass on the 512-patch workload split
over two ranks.
"""
import numpy as np
import pytest

import multirank as mr
from paper_2509_18261_gb300 import exchange as xch
from paper_2509_18261_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _ranks(params, batch, state, parts, first, n_ranks, launch):
    import torch

    from paper_2509_18261_gb300 import pmp

    rank_of = xch.partition(mr.positions(batch), mr.costs(batch, first), n_ranks)
    out = []
    for r in range(n_ranks):
        plan = xch.RankPlan(batch.dims, batch.nb, batch.g, rank_of, n_ranks, r)
        lb, st, lp, lf = mr.local_inputs(plan, batch, state, parts, first)
        rp = xch.RankPass(params, plan, torch.from_numpy(st).cuda(), pmp.parts_to_device(lp), lf, want_eta=True,
                          launch=launch)
        rp.lb, rp.first_np = lb, lf
        out.append(rp)
    return rank_of, out


def _exchange(ranks, kind):
    sent = [r.pack(kind) for r in ranks]
    for r in ranks:
        recv = r.msg[(kind, 0)]
        for peer, (a, b) in r.plan.layout[(kind, 0)][1].items():
            pa, pb = ranks[peer].plan.layout[(kind, 1)][1][r.plan.rank]
            assert pb - pa == b - a
            recv[a:b].copy_(sent[peer][pa:pb])
        r.unpack(kind)


def _run(ranks, kind):
    import torch

    from paper_2509_18261_gb300 import pmp

    _exchange(ranks, xch.STATE)
    for r in ranks:
        r.deposit()
    _exchange(ranks, xch.GHOST)
    if kind == "sink":
        _exchange(ranks, xch.FOLDED)
    for r in ranks:
        r.finish()
    torch.cuda.synchronize()
    for r in ranks:
        assert pmp.pmp_get_error(r.ctx) == (0, -1)


def _check(batch, first, ranks, want_state, want_eta, want_gathered, want_parts, kind):
    for rk in ranks:
        loc = rk.plan.local
        st = rk.state.cpu().numpy()
        eta = rk.eta.cpu().numpy()
        G = rk.gathered.cpu().numpy()
        parts = {k: v.cpu().numpy() for k, v in rk.parts.items()}
        v = 0
        for i in range(rk.plan.n_owned):
            gp = loc["global_id"][i]
            g = batch.g
            got = mr.local_view(rk.lb, st, i)[:, g:-g, g:-g, g:-g]
            assert np.array_equal(got.view(np.uint64), batch.valid(want_state, gp).view(np.uint64)), \
                f"state of patch {gp}"
            nv = int(batch.nvalid[gp])
            assert np.array_equal(eta[v:v + nv], want_eta[batch.vbase[gp]:batch.vbase[gp] + nv]), f"eta, patch {gp}"
            a, b = int(first[gp]), int(first[gp + 1])
            la = int(rk.first_np[i])
            assert np.array_equal(G[:, la:la + b - a].view(np.uint64), want_gathered[:, a:b].view(np.uint64)), \
                f"gathered rows of patch {gp}"
            if kind == "sink":
                for k in ("m", "px", "py", "pz"):
                    assert np.array_equal(parts[k][la:la + b - a], want_parts[k][a:b]), f"sink {k}, patch {gp}"
            v += nv


@pytest.mark.parametrize("launch", ["persistent", "per_patch"])
@pytest.mark.parametrize("kind", ["feedback", "sink"])
@pytest.mark.parametrize("n_ranks", [2, 3])
def test_decomposed_pass_matches_the_oracle(orc, kind, n_ranks, launch):
    rng, batch, state = mr.small_batch(5)
    if kind == "sink":
        for p in range(batch.np):
            v = batch.valid(state, p)
            v[0] *= 4.0
            v[4] *= 4.0
    parts, first = mr.boundary_particles(rng, batch, kind)
    params = syn.feedback_params() if kind == "feedback" else syn.sink_params(dt=4.0)
    ref_state, ref_parts = state.copy(), {k: v.copy() for k, v in parts.items()}
    ref = orc.batch_cycle(params, batch, ref_state, ref_parts, first, want_eta=True)
    _, ranks = _ranks(params, batch, state, parts, first, n_ranks, launch)
    _run(ranks, kind)
    _check(batch, first, ranks, ref_state, ref["eta"], ref["gathered"], ref_parts, kind)
    for r in ranks:
        r.close()


@pytest.mark.parametrize("kind", ["feedback", "sink"])
def test_512_patches_over_two_ranks_match_the_one_rank_pass(kind):
    import torch

    from paper_2509_18261_gb300 import pmp

    w = syn.make_batch_workload()
    batch, state = w["batch"], w["state"]
    parts, first = (w["fb"], w["fb_first"]) if kind == "feedback" else (w["sink"], w["sink_first"])
    params = w["fb_params"] if kind == "feedback" else w["sink_params"]
    one = pmp.BatchPass(params, batch, torch.from_numpy(state.copy()).cuda(), pmp.parts_to_device(parts), first,
                        want_eta=True)
    one.run("persistent")
    torch.cuda.synchronize()
    want_state = one.state.cpu().numpy()
    want_eta = one.eta.cpu().numpy()
    want_gathered = one.gathered_view().cpu().numpy()
    want_parts = {k: v.cpu().numpy() for k, v in one.parts.items()}
    one.close()
    rank_of, ranks = _ranks(params, batch, state, parts, first, 2, "persistent")
    assert set(rank_of) == {0, 1}
    _run(ranks, kind)
    _check(batch, first, ranks, want_state, want_eta, want_gathered, want_parts, kind)
    for r in ranks:
        r.close()
