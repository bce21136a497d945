"""The batched pass on several ranks: a domain decomposition of one level's
patches with the ghost-zone exchange of Sec. 2.2, Step 2 (the parts of a
buffer's ghost zones that lie on another rank's cells are sent to that rank
and added there in the fixed order of App. A.2).

Patches go to ranks along a space-filling curve (pmp_partition_sfc).  Each
rank keeps its owned patches plus one proxy per neighbouring patch of another
rank (pmp_plan_*), and one pass is

  STATE   exchange: neighbours' valid state cells into the proxies (the
          owned patches' ghost zones read them);
  part 1  Step 1 on the owned patches (pmp_cycle_batched_part, DEPOSIT);
  GHOST   exchange: each owned patch's buffer ghost cells that lie on a
          neighbour rank's cells go to that rank's proxy of the patch;
  FOLDED  exchange (sinks): folded sums next to the neighbours, for Step 4;
  part 2  Steps 2-5 on the owned patches (FINISH).

Packing and unpacking run in the library's kernels (pmp_batch_pack /
pmp_batch_unpack); the messages travel by torch.distributed point-to-point
sends and receives between neighbour ranks only (NCCL between GPUs, gloo on
the CPU).  There is no collective: the exchange is neighbour to neighbour.
The owned patches' results equal the one-rank batched pass bit for bit with
the deterministic (OWNER) deposit strategies, because every owned cell adds
the same images in the same order.
"""
from __future__ import annotations

import torch

from . import pmp

STATE, GHOST, FOLDED = pmp.XCH_STATE, pmp.XCH_GHOST, pmp.XCH_FOLDED
# device region list of each (exchange, send) pair in a batch
SLOTS = {(STATE, 1): 0, (STATE, 0): 1, (GHOST, 1): 2, (GHOST, 0): 3, (FOLDED, 1): 4, (FOLDED, 0): 5}


def partition(pos, cost, n_ranks):
    """Rank of every patch: the Morton curve of the super-grid positions
    `pos` (n, 3) cut into runs of about equal `cost`."""
    return pmp.pmp_partition_sfc(pos, cost, n_ranks)


def message_layout(regions):
    """(total doubles, {peer: (start, stop)}) of an exchange's region list."""
    spans = {}
    total = 0
    for r in regions:
        vol = 5 * (r["hi"][0] - r["lo"][0]) * (r["hi"][1] - r["lo"][1]) * (r["hi"][2] - r["lo"][2])
        a, b = r["offset"], r["offset"] + vol
        lo, hi = spans.get(r["peer"], (a, b))
        spans[r["peer"]] = (min(lo, a), max(hi, b))
        total = max(total, b)
    return total, spans


class RankPlan:
    """What one rank holds and exchanges (host only): the local patches and,
    for each exchange, the regions it sends and receives with their message
    layout."""

    def __init__(self, dims, nb, ng, rank_of, n_ranks, rank):
        self.rank, self.n_ranks, self.ng = rank, n_ranks, ng
        self.h = pmp.pmp_plan_create(dims, nb, ng, rank_of, n_ranks, rank)
        self.local = pmp.pmp_plan_local(self.h)
        self.regions = {key: pmp.pmp_plan_regions(self.h, key[0], key[1]) for key in SLOTS}
        self.layout = {key: message_layout(r) for key, r in self.regions.items()}

    @property
    def n_owned(self):
        return self.local["n_owned"]

    def close(self):
        self.h.close()


def p2p_exchange(send, recv, send_spans, recv_spans, group=None):
    """Sends send[start:stop] to every peer of send_spans and receives
    recv[start:stop] from every peer of recv_spans (torch.distributed
    point-to-point; peers are ranks of `group`)."""
    import torch.distributed as dist

    ops = []
    for peer, (a, b) in sorted(recv_spans.items()):
        if b > a:
            ops.append(dist.P2POp(dist.irecv, recv[a:b], peer, group))
    for peer, (a, b) in sorted(send_spans.items()):
        if b > a:
            ops.append(dist.P2POp(dist.isend, send[a:b], peer, group))
    if ops:
        # one group of sends and receives (NCCL: no ordering deadlock between peers)
        for r in dist.batch_isend_irecv(ops):
            r.wait()


class RankPass:
    """One rank's pass over its owned patches on its GPU: the local state
    arena (owned patches, proxies, zero patch; laid out as plan.local says),
    the owned patches' particles (patch after patch, `first` over all local
    patches with empty ranges for the others), a buffer arena, the gathered
    rows and the message buffers of the three exchanges."""

    def __init__(self, params, plan, state, parts, first, dx=1.0, want_eta=False, launch="persistent"):
        loc = plan.local
        self.plan, self.launch = plan, launch
        self.kind = params["kind"]
        self.ctx = pmp.Context(params)
        dev = state.device
        self.state = state
        self.buffer = torch.zeros(loc["arena_len"], dtype=torch.float64, device=dev)  # the zero patch stays zero
        self.parts = parts
        n = int(parts["x"].numel())
        self.n = n
        self.gathered = torch.zeros((pmp.pmp_gathered_rows(params["kind"]), max(n, 1)), dtype=torch.float64,
                                    device=dev)
        nvalid = sum(d[0] * d[1] * d[2] for d in loc["dims"][:loc["n_owned"]])
        self.eta = torch.empty(max(nvalid, 1), dtype=torch.float64, device=dev) if want_eta else None
        self.h = pmp.pmp_batch_create_partial(self.ctx, loc["dims"], loc["nb"], loc["offset"], loc["field_stride"],
                                              loc["n_owned"], plan.ng, loc["arena_len"], dx)
        pmp.pmp_batch_set_particles(self.h, first)
        for key, slot in SLOTS.items():
            pmp.pmp_batch_set_regions(self.h, slot, plan.regions[key])
        self.msg = {key: torch.zeros(max(plan.layout[key][0], 1), dtype=torch.float64, device=dev) for key in SLOTS}

    def kinds(self):
        """The exchanges of a pass of this kind, in order."""
        return (STATE, GHOST, FOLDED) if self.kind == "sink" else (STATE, GHOST)

    def pack(self, kind):
        arena = self.state if kind == STATE else self.buffer
        pmp.pmp_batch_pack(self.h, SLOTS[(kind, 1)], arena, self.msg[(kind, 1)], folded=kind == FOLDED)
        return self.msg[(kind, 1)]

    def unpack(self, kind):
        arena = self.state if kind == STATE else self.buffer
        pmp.pmp_batch_unpack(self.h, SLOTS[(kind, 0)], self.msg[(kind, 0)], arena)

    def deposit(self):
        pmp.pmp_cycle_batched_part(self.h, self.state, self.buffer, self.parts, self.gathered, self.eta,
                                   self.launch, pmp.PART_DEPOSIT)

    def finish(self):
        pmp.pmp_cycle_batched_part(self.h, self.state, self.buffer, self.parts, self.gathered, self.eta,
                                   self.launch, pmp.PART_FINISH)

    def exchange(self, kind, group=None):
        """Pack, send and receive, unpack one exchange (torch.distributed)."""
        send = self.pack(kind)
        p2p_exchange(send, self.msg[(kind, 0)], self.plan.layout[(kind, 1)][1], self.plan.layout[(kind, 0)][1],
                     group)
        self.unpack(kind)

    def run(self, group=None):
        """One pass: STATE, Step 1, GHOST (and FOLDED), Steps 2-5."""
        self.exchange(STATE, group)
        self.deposit()
        self.exchange(GHOST, group)
        if self.kind == "sink":
            self.exchange(FOLDED, group)
        self.finish()

    def gathered_view(self):
        return self.gathered[:, : self.n]

    def close(self):
        self.h.close()
        self.ctx.close()
