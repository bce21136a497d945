"""Seeded synthetic inputs shaped like the workloads of He et al. (2025), Sec. 4.

This module only draws random numbers and lays them out in memory; it holds
none of the particle-mesh-particle arithmetic.  Both the CUDA path and the CPU
oracle receive what it produces.

Recipe (the paper's own initial conditions, the AGORA disk of Sec. 4.6 and the
uniform Bondi/supernova boxes of Sec. 4.2-4.5, are not available, so these
stand in for them):

* gas: ln(rho) ~ N(-1/2, 1) (mean density 1); each momentum component
  ~ N(0, 0.1); total energy E = |p|^2/(2 rho) + rho * e_th with a uniform
  specific thermal energy e_th = 1 (uniform temperature).
* particle positions in cell units of the box, uniform in [0, n) per axis, or
  in Plummer clusters: radius a / sqrt(u^(-2/3) - 1) with u ~ U(0, 1), an
  isotropic direction, a uniform cluster centre, wrapped periodically.
* particle velocities ~ N(0, 0.1) per axis; momentum = mass * velocity.
* supernova (feedback) particles: ejecta mass log-uniform in [1e-3, 1e-1],
  supernova energy 1.0.
* sink particles: mass log-uniform in [1, 100].

Memory layout of a mesh: float64 array of shape (5, field_stride), field f at
row f; cell (i, j, k) of the padded box (nx+2g, ny+2g, nz+2g), x fastest.
``field_stride`` is the padded cell count rounded up to a multiple of 32
doubles (256 bytes) so that every field starts on a 256-byte boundary.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 2509_18261
NFIELDS = 5


@dataclasses.dataclass(frozen=True)
class Box:
    """A single box of ``n`` valid cells per axis with ``g`` ghost cells."""

    n: tuple
    g: int

    @property
    def padded(self):
        return tuple(m + 2 * self.g for m in self.n)

    @property
    def ncells_padded(self):
        px, py, pz = self.padded
        return px * py * pz

    @property
    def field_stride(self):
        c = self.ncells_padded
        return (c + 31) // 32 * 32

    @property
    def ncells_valid(self):
        return self.n[0] * self.n[1] * self.n[2]

    def grid(self, arr):
        """View (5, nz+2g, ny+2g, nx+2g) of a (5, field_stride) array."""
        px, py, pz = self.padded
        return arr[:, : self.ncells_padded].reshape(arr.shape[0], pz, py, px)

    def valid(self, arr):
        """View (5, nz, ny, nx) of the valid cells of a (5, field_stride) array."""
        g = self.g
        nx, ny, nz = self.n
        return self.grid(arr)[:, g : g + nz, g : g + ny, g : g + nx]

    def empty(self, fill=0.0):
        a = np.empty((NFIELDS, self.field_stride), dtype=np.float64)
        a.fill(fill)
        return a


def _uniform_positions(rng, count, n):
    pos = np.empty((3, count), dtype=np.float64)
    for a in range(3):
        p = rng.random(count) * n[a]
        # keep every coordinate strictly below n even after rounding
        np.minimum(p, np.nextafter(float(n[a]), 0.0), out=p)
        pos[a] = p
    return pos


def _plummer_positions(rng, nclusters, per_cluster, scale, n):
    count = nclusters * per_cluster
    centres = _uniform_positions(rng, nclusters, n)
    u = rng.random(count)
    u = np.clip(u, 1e-12, 1.0 - 1e-12)
    radius = scale / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
    d = rng.standard_normal((3, count))
    d /= np.sqrt((d * d).sum(axis=0))
    pos = np.empty((3, count), dtype=np.float64)
    for a in range(3):
        c = np.repeat(centres[a], per_cluster)
        p = np.mod(c + radius * d[a], float(n[a]))
        np.minimum(p, np.nextafter(float(n[a]), 0.0), out=p)
        p[p < 0.0] = 0.0
        pos[a] = p
    return pos


def gas_state(rng, box, ghost_fill=np.nan, e_th=1.0, sigma_p=0.1):
    """Lognormal gas with Gaussian momenta at uniform specific thermal energy.

    Ghost cells of the returned state hold ``ghost_fill`` (NaN by default):
    the library never reads or writes them.
    """
    u = box.empty(ghost_fill)
    v = box.valid(u)
    shape = v.shape[1:]
    rho = np.exp(rng.standard_normal(shape) - 0.5)
    px = rng.standard_normal(shape) * sigma_p
    py = rng.standard_normal(shape) * sigma_p
    pz = rng.standard_normal(shape) * sigma_p
    v[0] = rho
    v[1] = px
    v[2] = py
    v[3] = pz
    v[4] = (px * px + py * py + pz * pz) / (2.0 * rho) + rho * e_th
    return u


def uniform_gas(box, rho, vel=(0.0, 0.0, 0.0), e_th=1.0, ghost_fill=np.nan):
    """Uniform gas of density ``rho`` moving at ``vel`` (Bondi-type set-ups)."""
    u = box.empty(ghost_fill)
    v = box.valid(u)
    v[0] = rho
    for a in range(3):
        v[1 + a] = rho * vel[a]
    v[4] = 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2) + rho * e_th
    return u


def particles(rng, n, count, kind, clustered=0, nclusters=0, scale=2.0, sigma_v=0.1):
    """Particles of one kind: dict of float64 arrays x, y, z, m, px, py, pz, e.

    ``clustered`` of them sit in ``nclusters`` Plummer clusters of scale radius
    ``scale`` cells; the rest are uniform.  The order is shuffled so that the
    clusters interleave in index order.
    """
    nu = count - clustered
    parts = [_uniform_positions(rng, nu, n)]
    if clustered:
        assert clustered % nclusters == 0
        parts.append(_plummer_positions(rng, nclusters, clustered // nclusters, scale, n))
    pos = np.concatenate(parts, axis=1)
    perm = rng.permutation(count)
    pos = pos[:, perm]
    if kind == "feedback":
        m = np.exp(rng.uniform(math.log(1e-3), math.log(1e-1), count))
        e = np.ones(count)
    elif kind == "sink":
        m = np.exp(rng.uniform(math.log(1.0), math.log(100.0), count))
        e = np.zeros(count)
    else:
        raise ValueError(kind)
    vel = rng.standard_normal((3, count)) * sigma_v
    return {
        "x": np.ascontiguousarray(pos[0]),
        "y": np.ascontiguousarray(pos[1]),
        "z": np.ascontiguousarray(pos[2]),
        "m": m,
        "px": m * vel[0],
        "py": m * vel[1],
        "pz": m * vel[2],
        "e": e,
    }


def split_particles(p, idx):
    return {k: np.ascontiguousarray(v[idx]) for k, v in p.items()}


# --- parameter sets (code units; the values each workload uses) -------------

def mass_params(**kw):
    """Particle-mesh (PM/PIC) deposit: Steps 1, 2 and 5 of Sec. 2.2 with the
    supernova kernel (r_K = 2, S = 4 sub-points per axis)."""
    p = feedback_params(kind="mass")
    p.update(kw)
    return p


def feedback_params(**kw):
    p = dict(
        kind="feedback",
        r_K=2.0,
        subsample=4,
        dt=0.0,
        G=0.0,
        gamma=5.0 / 3.0,
        lambda_bh=0.0,
        J=0.25,
        cap=0.25,
        rho_min=0.0,
        A_sf=30.0,
        # P_snr^2 / (2 M_sf(n_H = 1)) = 0.46 E_sn (Sec. 3.2.1's 4.6e50 erg with
        # P_snr = 2.8e5 Msun km/s and M_sf = 1679 Msun); in code units M_sf(1) = A_sf
        A_p=math.sqrt(2.0 * 0.46 * 30.0),
        mu_H=1.0,
        RM_ej=0.027,
        RM_st=1.0,
        eps_K=0.28,
    )
    p.update(kw)
    return p


def sink_params(**kw):
    p = dict(
        kind="sink",
        r_K=4.0,
        subsample=1,
        dt=0.1,
        G=0.035,
        gamma=5.0 / 3.0,
        lambda_bh=math.exp(1.5) / 4.0,
        J=0.25,
        cap=0.25,
        rho_min=1e-6,
        A_sf=0.0,
        A_p=0.0,
        mu_H=1.0,
        RM_ej=0.027,
        RM_st=1.0,
        eps_K=0.28,
    )
    p.update(kw)
    return p


# --- the workloads ------------------------------------------------------------

WORKLOADS = {
    # name: (n, g, feedback spec, sink spec)
    "c1_32": dict(n=32, g=4, fb=dict(count=64), sink=dict(count=8)),
    "c2_256": dict(n=256, g=4, fb=dict(count=1_048_576, clustered=524_288, nclusters=32)),
    "c4_128": dict(n=128, g=4, fb=dict(count=262_144, clustered=131_072, nclusters=32)),
    "c5_512": dict(
        n=512,
        g=4,
        mixed=dict(count=16_777_216, clustered=4_194_304, nclusters=256, sink_fraction=8),
    ),
}

WORKLOAD_INDEX = {"c1_32": 0, "c2_256": 1, "c3_batched": 2, "c4_128": 3, "c5_512": 4}


def make_workload(name, n=None, count_scale=1.0, ghost_fill=np.nan, keep_cluster_size=False):
    """Build the named workload (optionally shrunk to box ``n``, counts scaled).

    With counts scaled, the clusters keep their number and shrink, or with
    ``keep_cluster_size`` keep their size and become fewer.  Returns
    dict(box, state, fb, sink, fb_params, sink_params); ``fb`` / ``sink`` are
    None when the workload has no particles of that kind.
    """
    spec = WORKLOADS[name]
    rng = np.random.default_rng(SEED_BASE + WORKLOAD_INDEX[name])
    nn = spec["n"] if n is None else n
    box = Box((nn, nn, nn), spec["g"])
    state = gas_state(rng, box, ghost_fill=ghost_fill)
    fb = sink = None

    def scaled(c):
        return max(1, int(round(c * count_scale)))

    if "fb" in spec:
        f = spec["fb"]
        cnt = scaled(f["count"])
        cl = 0
        if f.get("clustered"):
            ncl = f["nclusters"]
            cl = scaled(f["clustered"]) // ncl * ncl
        fb = particles(rng, box.n, cnt, "feedback", clustered=cl, nclusters=f.get("nclusters", 0))
    if "sink" in spec:
        sink = particles(rng, box.n, scaled(spec["sink"]["count"]), "sink")
    if "mixed" in spec:
        f = spec["mixed"]
        cnt = scaled(f["count"])
        ncl = f["nclusters"]
        if keep_cluster_size:
            size = f["clustered"] // ncl
            ncl = max(1, int(round(ncl * count_scale)))
            cl = ncl * size
        else:
            cl = scaled(f["clustered"]) // ncl * ncl
        allp = particles(rng, box.n, cnt, "feedback", clustered=cl, nclusters=ncl)
        nsink = cnt // f["sink_fraction"]
        fb = split_particles(allp, np.arange(0, cnt - nsink))
        sink = split_particles(allp, np.arange(cnt - nsink, cnt))
        sm = np.exp(rng.uniform(math.log(1.0), math.log(100.0), nsink))
        vel = rng.standard_normal((3, nsink)) * 0.1
        sink["m"] = sm
        sink["px"], sink["py"], sink["pz"] = sm * vel[0], sm * vel[1], sm * vel[2]
        sink["e"] = np.zeros(nsink)
    return dict(
        box=box,
        state=state,
        fb=fb,
        sink=sink,
        fb_params=feedback_params(),
        sink_params=sink_params(),
    )


# --- batched patches ----------------------------------------------------------

# Neighbour offsets (ox, oy, oz) of a patch, in the table order: oz slowest,
# ox fastest, the zero offset left out.
NB_OFFSETS = tuple(
    (ox, oy, oz) for oz in (-1, 0, 1) for oy in (-1, 0, 1) for ox in (-1, 0, 1) if (ox, oy, oz) != (0, 0, 0)
)


class Batch:
    """Patches of one level tiling a periodic rectilinear super-grid.

    ``edges = (sx, sy, sz)``: the x extent of every patch in super-column I is
    sx[I] (likewise y, z), so the patches tile a periodic box of
    (sum sx, sum sy, sum sz) cells.  Patch p = (K * P1 + J) * P0 + I.  Each
    patch keeps [5][field_stride] doubles (padded by g, stride rounded up to 32
    doubles) at ``offset[p]`` of one arena; ``nb[p]`` lists the patch displaced
    by each of NB_OFFSETS (periodically).
    """

    def __init__(self, edges, g):
        self.edges = tuple(tuple(int(v) for v in e) for e in edges)
        self.g = int(g)
        P0, P1, P2 = (len(e) for e in self.edges)
        self.sgrid = (P0, P1, P2)
        self.np = P0 * P1 * P2
        self.dims = np.zeros((self.np, 3), dtype=np.int32)
        self.origin = np.zeros((self.np, 3), dtype=np.int64)
        self.nb = np.zeros((self.np, 26), dtype=np.int32)
        starts = [np.concatenate([[0], np.cumsum(e)[:-1]]) for e in self.edges]
        for K in range(P2):
            for J in range(P1):
                for I in range(P0):
                    p = (K * P1 + J) * P0 + I
                    self.dims[p] = (self.edges[0][I], self.edges[1][J], self.edges[2][K])
                    self.origin[p] = (starts[0][I], starts[1][J], starts[2][K])
                    for t, (ox, oy, oz) in enumerate(NB_OFFSETS):
                        self.nb[p, t] = (((K + oz) % P2) * P1 + (J + oy) % P1) * P0 + (I + ox) % P0
        self.boxes = [Box(tuple(int(v) for v in self.dims[p]), self.g) for p in range(self.np)]
        self.fstride = np.array([b.field_stride for b in self.boxes], dtype=np.int64)
        self.offset = np.concatenate([[0], np.cumsum(NFIELDS * self.fstride)[:-1]]).astype(np.int64)
        self.arena_len = int(self.offset[-1] + NFIELDS * self.fstride[-1])
        self.nvalid = np.array([b.ncells_valid for b in self.boxes], dtype=np.int64)
        self.vbase = np.concatenate([[0], np.cumsum(self.nvalid)]).astype(np.int64)
        self.global_n = tuple(int(sum(e)) for e in self.edges)

    @property
    def ncells_valid(self):
        return int(self.vbase[-1])

    @property
    def ncells_padded(self):
        return int(sum(b.ncells_padded for b in self.boxes))

    def empty(self, fill=0.0):
        a = np.empty(self.arena_len, dtype=np.float64)
        a.fill(fill)
        return a

    def view(self, arena, p):
        """(5, field_stride) view of patch p in an arena."""
        o, fs = int(self.offset[p]), int(self.fstride[p])
        return arena[o : o + NFIELDS * fs].reshape(NFIELDS, fs)

    def grid(self, arena, p):
        return self.boxes[p].grid(self.view(arena, p))

    def valid(self, arena, p):
        return self.boxes[p].valid(self.view(arena, p))

    def to_global(self, arena):
        """The valid cells of all patches assembled into (5, Nz, Ny, Nx)."""
        Nx, Ny, Nz = self.global_n
        out = np.empty((NFIELDS, Nz, Ny, Nx), dtype=arena.dtype)
        for p in range(self.np):
            (x0, y0, z0), (nx, ny, nz) = self.origin[p], self.dims[p]
            out[:, z0 : z0 + nz, y0 : y0 + ny, x0 : x0 + nx] = self.valid(arena, p)
        return out

    def from_global(self, glob, fill=np.nan):
        """An arena whose valid cells are taken from a (5, Nz, Ny, Nx) array."""
        a = self.empty(fill)
        for p in range(self.np):
            (x0, y0, z0), (nx, ny, nz) = self.origin[p], self.dims[p]
            self.valid(a, p)[...] = glob[:, z0 : z0 + nz, y0 : y0 + ny, x0 : x0 + nx]
        return a


def batch_gas_state(rng, batch, ghost_fill=np.nan):
    """gas_state drawn patch after patch into one arena (ghosts = ghost_fill)."""
    a = batch.empty(ghost_fill)
    for p in range(batch.np):
        batch.view(a, p)[...] = gas_state(rng, batch.boxes[p], ghost_fill=ghost_fill)
    return a


def power_law_counts(rng, npatch, xmax=20001.0):
    """Per-patch counts n = floor(X) - 1 with density of X proportional to
    X^-2 on [1, xmax) (inverse transform sampling)."""
    u = rng.random(npatch)
    x = 1.0 / (1.0 - u * (1.0 - 1.0 / xmax))
    return np.floor(x).astype(np.int64) - 1


def concat_particles(chunks):
    keys = ("x", "y", "z", "m", "px", "py", "pz", "e")
    return {k: np.ascontiguousarray(np.concatenate([c[k] for c in chunks])) for k in keys}


def batch_particles(rng, batch, counts, kind):
    """Particles of one kind, uniform in each patch (patch-local cell units),
    stored patch after patch; returns (particles, first) with first[np] = total."""
    chunks = [particles(rng, batch.boxes[p].n, int(counts[p]), kind) for p in range(batch.np)]
    first = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return concat_particles(chunks), first


BATCH_EDGES = (16, 24, 32, 48, 64)


def make_batch_workload(supergrid=(8, 8, 8), edges=BATCH_EDGES, g=4, xmax=20001.0, sink_fraction=8, seed=None):
    """Uneven AMR-like patches: per super-column edges drawn uniformly from
    ``edges`` on each axis independently, lognormal gas, per-patch particle
    counts from power_law_counts, each particle a sink with probability
    1/sink_fraction, else a supernova.  Returns dict(batch, state, fb, fb_first,
    sink, sink_first, fb_params, sink_params)."""
    rng = np.random.default_rng(SEED_BASE + WORKLOAD_INDEX["c3_batched"] if seed is None else seed)
    ed = tuple(tuple(int(v) for v in rng.choice(edges, size=supergrid[a])) for a in range(3))
    batch = Batch(ed, g)
    state = batch_gas_state(rng, batch)
    total = power_law_counts(rng, batch.np, xmax)
    nsk = rng.binomial(total, 1.0 / sink_fraction)
    fb, fb_first = batch_particles(rng, batch, total - nsk, "feedback")
    sk, sk_first = batch_particles(rng, batch, nsk, "sink")
    return dict(batch=batch, state=state, fb=fb, fb_first=fb_first, sink=sk, sink_first=sk_first,
                fb_params=feedback_params(), sink_params=sink_params())
