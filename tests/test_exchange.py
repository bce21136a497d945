"""The batched pass on several ranks (the ghost-zone exchange of Sec. 2.2,
Step 2, across a domain decomposition; App. A.2's fixed order), on the CPU:

- the partition follows the Morton curve of the patches' super-grid places
  and balances their cost;
- every plan's send lists are, region for region, what the peer receives;
- a proxy stands for every other rank's patch next to an owned one;
- the pass decomposed over 2, 3 and 4 ranks -- each rank's two parts
  computed by the oracle on its local patches, the STATE, GHOST and (sinks)
  FOLDED exchanges packed and unpacked from the plan's region lists -- gives
  the one-rank batched pass of the oracle bit for bit: gathered rows, state,
  eta, sink masses and momenta; with particles on patch faces, edges and
  corners, next to other ranks' patches;
- the same over two gloo ranks with the library's point-to-point transport.
"""
import os

import numpy as np
import pytest

import multirank as mr
from paper_2509_18261_gb300 import exchange as xch
from paper_2509_18261_gb300 import synthetic as syn

KINDS = ("feedback", "sink")


def _params(kind):
    return syn.feedback_params() if kind == "feedback" else syn.sink_params(dt=4.0)


def _workload(kind, seed=5):
    rng, batch, state = mr.small_batch(seed)
    if kind == "sink":
        for p in range(batch.np):  # dense gas: the limiter acts next to patch faces
            v = batch.valid(state, p)
            v[0] *= 4.0
            v[4] *= 4.0
    parts, first = mr.boundary_particles(rng, batch, kind)
    return batch, state, parts, first


def _plans(batch, first, n_ranks):
    rank_of = xch.partition(mr.positions(batch), mr.costs(batch, first), n_ranks)
    return rank_of, [xch.RankPlan(batch.dims, batch.nb, batch.g, rank_of, n_ranks, r) for r in range(n_ranks)]


def test_partition_follows_the_morton_curve_and_balances_cost():
    rng, batch, _ = mr.small_batch(1, supergrid=(4, 4, 4))
    parts, first = mr.boundary_particles(rng, batch, "feedback", per_patch=3)
    pos, cost = mr.positions(batch), mr.costs(batch, first)

    def morton(p):
        k = 0
        for b in range(10):
            for a in range(3):
                k |= ((pos[p][a] >> b) & 1) << (3 * b + a)
        return k

    for n in (1, 2, 3, 5, 8):
        rank_of = xch.partition(pos, cost, n)
        order = sorted(range(batch.np), key=lambda p: (morton(p), p))
        ranks = [rank_of[p] for p in order]
        assert ranks == sorted(ranks), "contiguous runs of the curve"
        assert set(ranks) == set(range(n))
        share = sum(cost) / n
        loads = [sum(c for c, r in zip(cost, rank_of) if r == k) for k in range(n)]
        assert max(loads) <= share + max(cost)
        # each cut sits at the patch boundary nearest to k/n of the total:
        # between the two patches whose cost midpoints straddle it
        c = [cost[p] for p in order]
        mids = np.cumsum(c) - 0.5 * np.asarray(c, dtype=float)
        for k in range(1, n):
            s = ranks.index(k)
            assert mids[s - 1] < k * share <= mids[s], (n, k)


def test_partition_leaves_a_patch_for_every_rank():
    """A patch that carries most of the cost takes one rank; the ranks after
    it still get a patch each while there are patches left."""
    pos = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0), (0, 0, 1), (1, 0, 1)]
    for cost, n in (([1000, 1, 1, 1], 4), ([1, 1000, 1, 1, 1, 1], 5), ([1, 1, 1, 1, 1, 5000], 3)):
        rank_of = xch.partition(pos[:len(cost)], cost, n)
        ranks = list(rank_of)  # Morton order is index order here
        assert ranks == sorted(ranks) and set(ranks) == set(range(n)), (cost, n, ranks)


@pytest.mark.parametrize("n_ranks", [2, 3, 4])
def test_plans_send_what_the_peers_receive(n_ranks):
    batch, _, _, first = _workload("feedback")
    rank_of, plans = _plans(batch, first, n_ranks)
    for r, pr in enumerate(plans):
        loc = pr.local
        owned = [g for g in loc["global_id"][:pr.n_owned]]
        assert owned == [p for p in range(batch.np) if rank_of[p] == r]
        proxies = loc["global_id"][pr.n_owned:-1]
        remote = sorted({int(batch.nb[p][t]) for p in owned for t in range(26)} - set(owned))
        assert proxies == remote
        zero = len(loc["dims"]) - 1
        assert loc["global_id"][zero] == -1
        assert tuple(loc["dims"][zero]) == tuple(int(v) for v in batch.dims.max(axis=0))
        for i in range(pr.n_owned, zero + 1):
            assert set(loc["nb"][i]) == {zero}
        for kind in (xch.STATE, xch.GHOST, xch.FOLDED):
            for s, ps in enumerate(plans):
                if s == r:
                    continue
                mine = [x for x in pr.regions[(kind, 1)] if x["peer"] == s]
                theirs = [x for x in ps.regions[(kind, 0)] if x["peer"] == r]
                assert len(mine) == len(theirs)
                base_m = pr.layout[(kind, 1)][1].get(s, (0, 0))[0]
                base_t = ps.layout[(kind, 0)][1].get(r, (0, 0))[0]
                for a, b in zip(mine, theirs):
                    assert pr.local["global_id"][a["patch"]] == ps.local["global_id"][b["patch"]]
                    assert a["lo"] == b["lo"] and a["hi"] == b["hi"]
                    assert a["offset"] - base_m == b["offset"] - base_t


@pytest.mark.parametrize("n_ranks,tiny", [(2, False), (3, False), (4, False), (2, True)])
def test_plans_send_each_needed_box_once(n_ranks, tiny):
    """A plan moves no more than the pass needs: STATE and FOLDED regions lie
    in a patch's valid cells, GHOST regions in its ghost shell only, and no
    box appears twice in a list.  `tiny`: two 4-cell patches with 4 ghost
    cells side by side, where a neighbour's boxes for offsets -1, 0 and +1
    along an axis coincide."""
    if tiny:
        _, batch, _ = mr.small_batch(1, supergrid=(2, 1, 1), edges=(4,), g=4)
        first = np.zeros(batch.np + 1, dtype=np.int64)
    else:
        batch, _, _, first = _workload("feedback")
    _, plans = _plans(batch, first, n_ranks)
    seen = 0
    for pr in plans:
        for kind in (xch.STATE, xch.GHOST, xch.FOLDED):
            for side in (0, 1):
                regs = pr.regions[(kind, side)]
                keys = [(x["peer"], x["patch"], tuple(x["lo"]), tuple(x["hi"])) for x in regs]
                assert len(keys) == len(set(keys)), (kind, side)
                for x in regs:
                    n = [int(v) for v in pr.local["dims"][x["patch"]]]
                    lo, hi = list(x["lo"]), list(x["hi"])
                    assert all(l < h for l, h in zip(lo, hi))
                    inside = [0 <= l and h <= na for l, h, na in zip(lo, hi, n)]
                    if kind == xch.GHOST:
                        assert not all(inside), "a GHOST region reaches into valid cells"
                        assert all(lo[a] >= n[a] or hi[a] <= 0 or inside[a] for a in range(3))
                    else:
                        assert all(inside), "a STATE or FOLDED region reaches into ghost cells"
                    seen += 1
    assert seen > 0


def _compare(orc, kind, batch, state, parts, first, ranks, rank_of):
    params = _params(kind)
    ref_state = state.copy()
    ref_parts = {k: v.copy() for k, v in parts.items()}
    ref = orc.batch_cycle(params, batch, ref_state, ref_parts, first, want_eta=True)
    for rk in ranks:
        loc = rk.plan.local
        v = 0
        for i in range(rk.plan.n_owned):
            gp = loc["global_id"][i]
            got = mr.local_view(rk.lb, rk.state, i)[:, batch.g:-batch.g, batch.g:-batch.g, batch.g:-batch.g]
            want = batch.valid(ref_state, gp)
            assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), f"state of patch {gp}"
            nv = int(batch.nvalid[gp])
            assert np.array_equal(rk.eta[v:v + nv], ref["eta"][batch.vbase[gp]:batch.vbase[gp] + nv])
            a, b = int(first[gp]), int(first[gp + 1])
            la = int(rk.first[i])
            assert np.array_equal(rk.gathered[:, la:la + b - a].view(np.uint64),
                                  ref["gathered"][:, a:b].view(np.uint64)), f"gathered rows of patch {gp}"
            if kind == "sink":
                for k in ("m", "px", "py", "pz"):
                    assert np.array_equal(rk.parts[k][la:la + b - a], ref_parts[k][a:b]), f"sink {k}, patch {gp}"
            v += nv
    return ref


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n_ranks", [2, 3, 4])
def test_decomposed_pass_equals_the_one_rank_pass(orc, kind, n_ranks):
    batch, state, parts, first = _workload(kind)
    params = _params(kind)
    rank_of, plans = _plans(batch, first, n_ranks)
    ranks = [mr.OracleRank(orc, params, pl, batch, state, parts, first) for pl in plans]
    mr.exchange_in_process(ranks, xch.STATE)
    for r in ranks:
        r.deposit()
    mr.exchange_in_process(ranks, xch.GHOST)
    if kind == "sink":
        mr.exchange_in_process(ranks, xch.FOLDED)
    for r in ranks:
        r.finish()
    ref = _compare(orc, kind, batch, state, parts, first, ranks, rank_of)
    if kind == "sink":
        assert ref["counts"][0] > 0  # the limiter acted


@pytest.mark.parametrize("supergrid,n_ranks", [((1, 2, 3), 2), ((2, 2, 2), 3), ((2, 1, 1), 2), ((3, 1, 2), 3)])
@pytest.mark.parametrize("kind", KINDS)
def test_decomposition_of_thin_super_grids(orc, kind, supergrid, n_ranks):
    """Super-grids one or two patches wide: a patch is its own neighbour
    across an axis, or the same remote patch is the neighbour on both sides
    (two different slabs of one proxy)."""
    rng, batch, state = mr.small_batch(11 + sum(supergrid), supergrid=supergrid)
    if kind == "sink":
        for p in range(batch.np):
            v = batch.valid(state, p)
            v[0] *= 4.0
            v[4] *= 4.0
    parts, first = mr.boundary_particles(rng, batch, kind)
    params = _params(kind)
    rank_of, plans = _plans(batch, first, n_ranks)
    ranks = [mr.OracleRank(orc, params, pl, batch, state, parts, first) for pl in plans]
    mr.exchange_in_process(ranks, xch.STATE)
    for r in ranks:
        r.deposit()
    mr.exchange_in_process(ranks, xch.GHOST)
    if kind == "sink":
        mr.exchange_in_process(ranks, xch.FOLDED)
    for r in ranks:
        r.finish()
    _compare(orc, kind, batch, state, parts, first, ranks, rank_of)


def _gloo_rank(rank, world, port, kind, out_dir):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle

        batch, state, parts, first = _workload(kind)
        _, plans = _plans(batch, first, world)
        rk = mr.OracleRank(oracle, _params(kind), plans[rank], batch, state, parts, first)

        def exchange(k):
            total, spans = rk.plan.layout[(k, 0)]
            send = torch.from_numpy(rk.pack(k))
            recv = torch.zeros(max(total, 1), dtype=torch.float64)
            xch.p2p_exchange(send, recv, rk.plan.layout[(k, 1)][1], spans)
            rk.unpack(k, recv.numpy())

        exchange(xch.STATE)
        rk.deposit()
        exchange(xch.GHOST)
        if kind == "sink":
            exchange(xch.FOLDED)
        rk.finish()
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), state=rk.state, eta=rk.eta, gathered=rk.gathered,
                 **{f"p_{k}": v for k, v in rk.parts.items()})
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("kind", KINDS)
def test_gloo_ranks_equal_the_one_rank_pass(orc, kind, world, tmp_path):
    """With three ranks a rank exchanges with two peers at once, one message
    per peer in each buffer."""
    import socket

    import torch.multiprocessing as tmp

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    tmp.spawn(_gloo_rank, args=(world, port, kind, str(tmp_path)), nprocs=world, join=True)
    batch, state, parts, first = _workload(kind)
    rank_of, plans = _plans(batch, first, world)
    ranks = []
    for r in range(world):
        d = np.load(tmp_path / f"rank{r}.npz")
        rk = mr.OracleRank(orc, _params(kind), plans[r], batch, state, parts, first)
        rk.state, rk.eta, rk.gathered = d["state"], d["eta"], d["gathered"]
        rk.parts = {k: d[f"p_{k}"] for k in rk.parts}
        ranks.append(rk)
    _compare(orc, kind, batch, state, parts, first, ranks, rank_of)
