"""Helpers of the multi-rank tests: a batch of uneven patches decomposed over
ranks with the library's partition and plan (host calls of libpmp), each
rank's part of the pass computed by the oracle on its local patches
(owned + proxies + zero patch), the exchanges packed and unpacked from the
plan's region lists.

Proxy state cells that no exchange fills are NaN, so a read of a cell the
plan forgot shows up in the results."""
from types import SimpleNamespace

import numpy as np

from paper_2509_18261_gb300 import exchange as xch
from paper_2509_18261_gb300 import synthetic as syn


def positions(batch):
    """Super-grid position (I, J, K) of every patch (patch p = (K P1 + J) P0 + I)."""
    P0, P1, _ = batch.sgrid
    return [(p % P0, (p // P0) % P1, p // (P0 * P1)) for p in range(batch.np)]


def costs(batch, first, weight=64):
    return [int(batch.nvalid[p]) + weight * int(first[p + 1] - first[p]) for p in range(batch.np)]


def local_batch(plan):
    """A batch-like view of a rank's local patches for the oracle."""
    loc = plan.local
    n = len(loc["dims"])
    return SimpleNamespace(
        np=n, g=plan.ng,
        dims=np.array(loc["dims"], dtype=np.int32), nb=np.array(loc["nb"], dtype=np.int32),
        offset=np.array(loc["offset"], dtype=np.int64), fstride=np.array(loc["field_stride"], dtype=np.int64),
        boxes=[syn.Box(tuple(int(v) for v in loc["dims"][i]), plan.ng) for i in range(n)],
        arena_len=int(loc["arena_len"]))


def local_view(lb, arena, i):
    o, fs = int(lb.offset[i]), int(lb.fstride[i])
    return lb.boxes[i].grid(arena[o:o + 5 * fs].reshape(5, fs))


def local_inputs(plan, batch, state, parts, first):
    """Local state arena (owned patches from the global arena, proxies NaN,
    the zero patch zero), the owned particles and their ranges."""
    loc = plan.local
    lb = local_batch(plan)
    st = np.full(lb.arena_len, np.nan)
    keys = ("x", "y", "z", "m", "px", "py", "pz", "e")
    chunks, lfirst = [], [0]
    for i, gp in enumerate(loc["global_id"]):
        if gp < 0:
            local_view(lb, st, i)[...] = 0.0
        if i < loc["n_owned"]:
            local_view(lb, st, i)[...] = batch.grid(state, gp)
            a, b = int(first[gp]), int(first[gp + 1])
            chunks.append({k: parts[k][a:b] for k in keys})
            lfirst.append(lfirst[-1] + b - a)
        else:
            lfirst.append(lfirst[-1])
    lparts = {k: np.ascontiguousarray(np.concatenate([c[k] for c in chunks]) if chunks else np.zeros(0))
              for k in keys}
    return lb, st, lparts, np.array(lfirst, dtype=np.int64)


def pack(lb, regions, arena, total):
    msg = np.zeros(max(total, 1))
    for r in regions:
        g = lb.g
        v = local_view(lb, arena, r["patch"])
        (x0, y0, z0), (x1, y1, z1) = r["lo"], r["hi"]
        blk = v[:, z0 + g:z1 + g, y0 + g:y1 + g, x0 + g:x1 + g].reshape(-1)
        msg[r["offset"]:r["offset"] + blk.size] = blk
    return msg


def unpack(lb, regions, msg, arena):
    for r in regions:
        g = lb.g
        v = local_view(lb, arena, r["patch"])
        (x0, y0, z0), (x1, y1, z1) = r["lo"], r["hi"]
        shape = (5, z1 - z0, y1 - y0, x1 - x0)
        n = int(np.prod(shape))
        v[:, z0 + g:z1 + g, y0 + g:y1 + g, x0 + g:x1 + g] = msg[r["offset"]:r["offset"] + n].reshape(shape)


class OracleRank:
    """One rank's pass computed by the oracle, step by step, so that a driver
    can run the exchanges between the steps (in one process, or over
    torch.distributed)."""

    def __init__(self, orc, params, plan, batch, state, parts, first):
        self.orc, self.params, self.plan = orc, params, plan
        self.lb, self.state, self.parts, self.first = local_inputs(plan, batch, state, parts, first)
        self.buf = np.zeros(self.lb.arena_len)
        n = int(self.first[-1])
        self.gathered = np.zeros((len(orc.rows(params["kind"])), n))
        nv = sum(int(np.prod(d)) for d in plan.local["dims"][:plan.n_owned])
        self.eta = np.zeros(max(nv, 1))

    def pack(self, kind):
        key = (kind, 1)
        total = self.plan.layout[key][0]
        if kind == xch.STATE:
            return pack(self.lb, self.plan.regions[key], self.state, total)
        if kind == xch.GHOST:
            return pack(self.lb, self.plan.regions[key], self.buf, total)
        folded = self.buf.copy()
        self.orc.batch_fold(self.lb, folded)  # owned cells: their App. A.2 sums
        return pack(self.lb, self.plan.regions[key], folded, total)

    def unpack(self, kind, msg):
        unpack(self.lb, self.plan.regions[(kind, 0)], msg, self.state if kind == xch.STATE else self.buf)

    def deposit(self):
        self.orc.batch_part(self.params, self.lb, self.plan.n_owned, 0, self.state, self.buf, self.parts,
                            self.first, self.gathered)

    def finish(self):
        self.counts = self.orc.batch_part(self.params, self.lb, self.plan.n_owned, 1, self.state, self.buf,
                                          self.parts, self.first, self.gathered, self.eta)


def exchange_in_process(ranks, kind):
    """Every rank packs; every rank receives its peers' messages (sliced by
    the plan's layouts) and unpacks."""
    sent = [r.pack(kind) for r in ranks]
    for r in ranks:
        total, spans = r.plan.layout[(kind, 0)]
        recv = np.zeros(max(total, 1))
        for peer, (a, b) in spans.items():
            pa, pb = ranks[peer].plan.layout[(kind, 1)][1][r.plan.rank]
            assert pb - pa == b - a, "message sizes agree"
            recv[a:b] = sent[peer][pa:pb]
        r.unpack(kind, recv)


def boundary_particles(rng, batch, kind, per_patch=6):
    """Particles on the faces, edges and corners of every patch (patch-local
    cell units), plus a few inside: a decomposition puts many of them next to
    another rank's patch."""
    chunks = []
    counts = []
    for p in range(batch.np):
        n = batch.dims[p]
        pts = []
        for _ in range(per_patch):
            x = [rng.uniform(0, n[a]) for a in range(3)]
            for a in rng.choice(3, size=rng.integers(1, 4), replace=False):
                x[a] = float(rng.choice([0.0, 0.25, np.nextafter(float(n[a]), 0.0), n[a] - 0.5, 1.75]))
            pts.append(x)
        pts = np.array(pts)
        m = np.exp(rng.uniform(np.log(1e-3), np.log(1e-1), per_patch)) if kind == "feedback" else \
            np.exp(rng.uniform(0.0, np.log(100.0), per_patch))
        v = rng.normal(0, 0.1, (3, per_patch))
        chunks.append(dict(x=pts[:, 0].copy(), y=pts[:, 1].copy(), z=pts[:, 2].copy(), m=m, px=m * v[0],
                           py=m * v[1], pz=m * v[2], e=np.ones(per_patch)))
        counts.append(per_patch)
    first = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return syn.concat_particles(chunks), first


def small_batch(seed, supergrid=(3, 3, 2), edges=(8, 12, 16), g=4):
    rng = np.random.default_rng(seed)
    ed = tuple(tuple(int(v) for v in rng.choice(edges, size=supergrid[a])) for a in range(3))
    batch = syn.Batch(ed, g)
    state = syn.batch_gas_state(rng, batch)
    return rng, batch, state
