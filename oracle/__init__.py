"""CPU oracle for the particle-mesh-particle cycle -- TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded FP64 restatement of He et al. (2025), Sec. 2.2
(Steps 1-5), Sec. 3.1.1 (sink accretion) and Sec. 3.2.1 (supernova feedback),
written in C (``pmp_oracle.c``) and driven from here through ctypes.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the library never does, and the two
share no code.

Functions take the (5, field_stride) float64 arrays and particle dicts that
``paper_2509_18261_gb300.synthetic`` produces, and mutate outputs in place
where the C function does.

Parity unpinned: the covered fraction omega (its sub-sampling rule) and the
code-unit constants A_sf, A_p have no printed values in the paper; they are
pinned only by self-consistency tests (conservation, symmetry, convergence).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pmp_oracle.c")
# PMP_ORACLE_LIB names a prebuilt oracle library to load instead of building
# this one: the pin-strength test (tests/test_oracle_mutants.py) builds copies
# of the oracle with planted mistakes and runs the pins against each.
_PREBUILT = os.environ.get("PMP_ORACLE_LIB")
_LIB = _PREBUILT or os.path.join(_HERE, "_build", "liboracle.so")

KIND = {"feedback": 0, "sink": 1, "mass": 2}
FB_ROWS = ["M_snr", "V_snr", "vcom_x", "vcom_y", "vcom_z", "n_H", "R_M", "p_rad", "q", "e", "Pv", "regime"]
SK_ROWS = ["rho_inf", "v_inf", "c_inf", "mdot", "r_acc", "sum_w", "K", "n_mem"]
MS_ROWS = ["V_K", "q_m", "q_px", "q_py", "q_pz", "q_e"]
STATUS = {0: "ok", 1: "bad argument", 2: "particle outside", 3: "non-finite", 4: "out of memory"}


class OracleError(RuntimeError):
    pass


def build(force=False):
    """Compile the oracle (no fused multiply-add, no fast-math)."""
    if _PREBUILT:
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = [
        "gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fexcess-precision=standard",
        "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm",
    ]
    subprocess.check_call(cmd)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("subsample", ctypes.c_int32),
        ("r_K", ctypes.c_double), ("dt", ctypes.c_double), ("G", ctypes.c_double),
        ("gamma", ctypes.c_double), ("lambda_bh", ctypes.c_double), ("J", ctypes.c_double),
        ("cap", ctypes.c_double), ("rho_min", ctypes.c_double), ("A_sf", ctypes.c_double),
        ("A_p", ctypes.c_double), ("mu_H", ctypes.c_double), ("RM_ej", ctypes.c_double),
        ("RM_st", ctypes.c_double), ("eps_K", ctypes.c_double),
    ]


class Mesh(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 3), ("ng", ctypes.c_int32), ("periodic", ctypes.c_int32 * 3),
        ("pad_", ctypes.c_int32), ("dx", ctypes.c_double), ("fstride", ctypes.c_int64),
        ("u", ctypes.POINTER(ctypes.c_double)),
    ]


class Particles(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_int64),
        ("x", ctypes.POINTER(ctypes.c_double)), ("y", ctypes.POINTER(ctypes.c_double)),
        ("z", ctypes.POINTER(ctypes.c_double)), ("m", ctypes.POINTER(ctypes.c_double)),
        ("px", ctypes.POINTER(ctypes.c_double)), ("py", ctypes.POINTER(ctypes.c_double)),
        ("pz", ctypes.POINTER(ctypes.c_double)), ("e", ctypes.POINTER(ctypes.c_double)),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        for name in ("or_exp", "or_log"):
            getattr(L, name).restype = ctypes.c_double
            getattr(L, name).argtypes = [ctypes.c_double]
        L.or_pow.restype = ctypes.c_double
        L.or_pow.argtypes = [ctypes.c_double, ctypes.c_double]
        L.or_bins_build.restype = ctypes.c_void_p
        L.or_bins_build.argtypes = [ctypes.POINTER(Mesh), ctypes.POINTER(Particles)]
        L.or_bins_free.argtypes = [ctypes.c_void_p]
        L.or_cells_at.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Mesh), ctypes.POINTER(Particles),
                                  ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                  dp, dp, dp, dp]
        L.or_sinks_at.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Mesh), ctypes.POINTER(Particles),
                                  ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, dp]
        L.or_gather_at.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Mesh), ctypes.POINTER(Particles),
                                   ctypes.c_int64, ctypes.c_void_p, dp]
        L.or_kernel_of.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Mesh), ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_void_p, dp]
        L.or_deltas.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Mesh), ctypes.POINTER(Particles), dp,
                                ctypes.c_void_p, dp]
        _lib = L
    return _lib


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_params(p):
    return Params(
        kind=KIND[p["kind"]], subsample=int(p["subsample"]), r_K=p["r_K"], dt=p["dt"], G=p["G"],
        gamma=p["gamma"], lambda_bh=p["lambda_bh"], J=p["J"], cap=p["cap"], rho_min=p["rho_min"],
        A_sf=p["A_sf"], A_p=p["A_p"], mu_H=p["mu_H"], RM_ej=p["RM_ej"], RM_st=p["RM_st"], eps_K=p["eps_K"],
    )


def make_mesh(box, arr, dx=1.0, periodic=(1, 1, 1)):
    assert arr.shape == (5, box.field_stride)
    return Mesh(n=(ctypes.c_int32 * 3)(*box.n), ng=box.g, periodic=(ctypes.c_int32 * 3)(*periodic),
                pad_=0, dx=dx, fstride=box.field_stride, u=_dp(arr))


def make_particles(p):
    for k in ("x", "y", "z", "m", "px", "py", "pz", "e"):
        assert p[k].dtype == np.float64 and p[k].flags["C_CONTIGUOUS"], k
    return Particles(count=len(p["x"]), x=_dp(p["x"]), y=_dp(p["y"]), z=_dp(p["z"]), m=_dp(p["m"]),
                     px=_dp(p["px"]), py=_dp(p["py"]), pz=_dp(p["pz"]), e=_dp(p["e"]))


def _check(st, what, strict=True):
    if st and strict:
        raise OracleError(f"{what}: {STATUS.get(st, st)}")
    return st


def rows(kind):
    return FB_ROWS if kind == "feedback" else (SK_ROWS if kind == "sink" else MS_ROWS)


def exp(x):
    return lib().or_exp(float(x))


def log(x):
    return lib().or_log(float(x))


def gather(params, box, state, parts, dx=1.0, periodic=(1, 1, 1), strict=True):
    """Gathered per-particle quantities, array [rows][count]."""
    P = make_params(params)
    n = len(parts["x"])
    G = np.zeros((len(rows(params["kind"])), n), dtype=np.float64)
    S = make_mesh(box, state, dx, periodic)
    pp = make_particles(parts)
    st = lib().or_gather(ctypes.byref(P), ctypes.byref(S), ctypes.byref(pp), _dp(G))
    _check(st, "gather", strict)
    return G


def deposit(params, box, state, parts, gathered, buf, absbuf=None, dx=1.0, periodic=(1, 1, 1), strict=True):
    """Step 1 into ``buf`` (and sum |dU| into ``absbuf``), in place."""
    P = make_params(params)
    S = make_mesh(box, state, dx, periodic)
    B = make_mesh(box, buf, dx, periodic)
    pp = make_particles(parts)
    st = lib().or_deposit(ctypes.byref(P), ctypes.byref(S), ctypes.byref(pp), _dp(gathered), ctypes.byref(B),
                          _dp(absbuf))
    return _check(st, "deposit", strict)


def deposit_rounded(params, box, state, parts, gathered, buf, M=28, dx=1.0, periodic=(1, 1, 1), strict=True):
    """Step 1 with the reproducible atomics of App. A.1 (index order): adds
    into ``buf``, then rounds every buffer value; returns the error bound E."""
    P = make_params(params)
    S = make_mesh(box, state, dx, periodic)
    B = make_mesh(box, buf, dx, periodic)
    pp = make_particles(parts)
    E = np.zeros_like(buf)
    st = lib().or_deposit_rounded(ctypes.byref(P), ctypes.byref(S), ctypes.byref(pp), _dp(gathered), ctypes.byref(B),
                                  int(M), _dp(E))
    _check(st, "deposit_rounded", strict)
    return E


def apply_extra(params, box, state, buf, extra, dx=1.0, periodic=(1, 1, 1)):
    """Auxiliary fields (n, field_stride) at fixed specific value under
    accretion, in place; call before the pass's apply."""
    P = make_params(params)
    S = make_mesh(box, state, dx, periodic)
    B = make_mesh(box, buf, dx, periodic)
    assert extra.dtype == np.float64 and extra.flags["C_CONTIGUOUS"] and extra.ndim == 2
    _check(lib().or_apply_extra(ctypes.byref(P), ctypes.byref(S), ctypes.byref(B), _dp(extra),
                                int(extra.shape[0]), ctypes.c_int64(extra.shape[1])), "apply_extra")


def create_sinks(params, box, state, buf, cap=None, dx=1.0, periodic=(1, 1, 1)):
    """Sink creation after an accretion pass (Sec. 3.1.2), ``state`` updated
    in place; returns (count, new sinks dict x, y, z, m, px, py, pz)."""
    P = make_params(params)
    S = make_mesh(box, state, dx, periodic)
    B = make_mesh(box, buf, dx, periodic)
    if cap is None:
        cap = box.ncells_valid
    out = {k: np.zeros(max(cap, 1)) for k in ("x", "y", "z", "m", "px", "py", "pz")}
    L = lib()
    L.or_create_sinks.restype = ctypes.c_int64
    n = L.or_create_sinks(ctypes.byref(P), ctypes.byref(S), ctypes.byref(B), ctypes.c_int64(cap),
                          *[_dp(out[k]) for k in ("x", "y", "z", "m", "px", "py", "pz")])
    if n < 0:
        raise OracleError("create_sinks failed")
    k = min(n, cap)
    return n, {key: v[:k].copy() for key, v in out.items()}


def fold(box, buf, absbuf=None, periodic=(1, 1, 1)):
    B = make_mesh(box, buf, 1.0, periodic)
    _check(lib().or_fold(ctypes.byref(B), _dp(absbuf)), "fold")


def return_sinks(params, box, state, buf, parts, gathered, dx=1.0, periodic=(1, 1, 1), strict=True):
    """Step 4 for sinks: parts['m'], parts['px'..'pz'] updated in place."""
    P = make_params(params)
    S = make_mesh(box, state, dx, periodic)
    B = make_mesh(box, buf, dx, periodic)
    pp = make_particles(parts)
    st = lib().or_return_sinks(ctypes.byref(P), ctypes.byref(S), ctypes.byref(B), ctypes.byref(pp), _dp(gathered))
    return _check(st, "return_sinks", strict)


def apply(params, box, state, buf, dx=1.0, periodic=(1, 1, 1), want_eta=False):
    """Steps 3 + 5 in place on ``state``; returns (eta or None, counts)."""
    P = make_params(params)
    S = make_mesh(box, state, dx, periodic)
    B = make_mesh(box, buf, dx, periodic)
    eta = np.empty(box.ncells_valid, dtype=np.float64) if want_eta else None
    counts = np.zeros(2, dtype=np.int64)
    st = lib().or_apply(ctypes.byref(P), ctypes.byref(S), ctypes.byref(B), _dp(eta),
                        counts.ctypes.data_as(ctypes.c_void_p))
    _check(st, "apply")
    return eta, counts


def cycle(params, box, state, parts, dx=1.0, periodic=(1, 1, 1), want_abs=False, want_eta=False):
    """One full pass (Steps 1-5; Step 4 for sinks).  Mutates ``state`` and, for
    sinks, the particle mass and momentum.  Returns a dict with the gathered
    rows, the folded buffer, the |dU| buffer, eta and limiter counts."""
    G = gather(params, box, state, parts, dx, periodic)
    buf = box.empty(0.0)
    absbuf = box.empty(0.0) if want_abs else None
    deposit(params, box, state, parts, G, buf, absbuf, dx, periodic)
    pre_fold = buf.copy()
    fold(box, buf, absbuf, periodic)
    if params["kind"] == "sink":
        return_sinks(params, box, state, buf, parts, G, dx, periodic)
    eta, counts = apply(params, box, state, buf, dx, periodic, want_eta=want_eta)
    return dict(gathered=G, buf=buf, pre_fold=pre_fold, absbuf=absbuf, eta=eta, counts=counts)


class Bins:
    """Particles binned by host cell, for one-by-one evaluation on big boxes."""

    def __init__(self, box, state, parts, dx=1.0, periodic=(1, 1, 1)):
        self.box, self.state, self.parts = box, state, parts
        self.dx, self.periodic = dx, periodic
        self._S = make_mesh(box, state, dx, periodic)
        self._p = make_particles(parts)
        self._h = lib().or_bins_build(ctypes.byref(self._S), ctypes.byref(self._p))
        if not self._h:
            raise OracleError("bins: out of memory")

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_bins_free(self._h)
            self._h = None

    def cells(self, params, ijk):
        """Summed buffer, |dU| sum, updated state and eta at valid cells ijk (n, 3)."""
        ijk = np.ascontiguousarray(ijk, dtype=np.int32)
        n = ijk.shape[0]
        s = np.empty((n, 5)); a = np.empty((n, 5)); u = np.empty((n, 5)); e = np.empty(n)
        P = make_params(params)
        st = lib().or_cells_at(ctypes.byref(P), ctypes.byref(self._S), ctypes.byref(self._p), self._h,
                               self.box.g, n, ijk.ctypes.data_as(ctypes.c_void_p), _dp(s), _dp(a), _dp(u), _dp(e))
        _check(st, "cells_at")
        return s, a, u, e

    def sinks(self, params, sel):
        """Updated (m, px, py, pz) of the listed sinks, array (n, 4)."""
        sel = np.ascontiguousarray(sel, dtype=np.int64)
        out = np.empty((len(sel), 4))
        P = make_params(params)
        st = lib().or_sinks_at(ctypes.byref(P), ctypes.byref(self._S), ctypes.byref(self._p), self._h,
                               self.box.g, len(sel), sel.ctypes.data_as(ctypes.c_void_p), _dp(out))
        _check(st, "sinks_at")
        return out

    def gather(self, params, sel):
        sel = np.ascontiguousarray(sel, dtype=np.int64)
        G = np.empty((len(rows(params["kind"])), len(sel)))
        P = make_params(params)
        st = lib().or_gather_at(ctypes.byref(P), ctypes.byref(self._S), ctypes.byref(self._p), len(sel),
                                sel.ctypes.data_as(ctypes.c_void_p), _dp(G))
        _check(st, "gather_at")
        return G


def kernel_of(params, box, x, y, z, periodic=(1, 1, 1)):
    """Kernel cells (unwrapped ijk, shape (n, 3)) and omega of a particle at (x, y, z)."""
    R = int(np.ceil(params["r_K"]))
    w = 2 * R + 1
    ijk = np.zeros((w ** 3, 3), dtype=np.int32)
    om = np.zeros(w ** 3)
    P = make_params(params)
    dummy = box.empty(0.0)
    S = make_mesh(box, dummy, 1.0, periodic)
    n = lib().or_kernel_of(ctypes.byref(P), ctypes.byref(S), x, y, z, ijk.ctypes.data_as(ctypes.c_void_p), _dp(om))
    return ijk[:n].copy(), om[:n].copy()


def deltas(params, box, state, one, dx=1.0, periodic=(1, 1, 1)):
    """Gathered row and Delta U^s of a single particle (dict of length-1
    arrays): returns (ijk (n, 3) unwrapped, dU (n, 5))."""
    G = gather(params, box, state, one, dx, periodic)
    R = int(np.ceil(params["r_K"]))
    w = 2 * R + 1
    ijk = np.zeros((w ** 3, 3), dtype=np.int32)
    dU = np.zeros((w ** 3, 5))
    P = make_params(params)
    S = make_mesh(box, state, dx, periodic)
    pp = make_particles(one)
    n = lib().or_deltas(ctypes.byref(P), ctypes.byref(S), ctypes.byref(pp), _dp(np.ascontiguousarray(G)),
                        ijk.ctypes.data_as(ctypes.c_void_p), _dp(dU))
    return ijk[:n].copy(), dU[:n].copy()


# --- batched patches ----------------------------------------------------------

class BatchT(ctypes.Structure):
    _fields_ = [
        ("np", ctypes.c_int32), ("ng", ctypes.c_int32), ("dx", ctypes.c_double),
        ("dims", ctypes.c_void_p), ("nb", ctypes.c_void_p), ("offset", ctypes.c_void_p),
        ("fstride", ctypes.c_void_p), ("first", ctypes.c_void_p),
    ]


def _batch_struct(batch, first, dx=1.0):
    """ctypes view of a synthetic.Batch (arrays kept alive by the caller)."""
    keep = dict(
        dims=np.ascontiguousarray(batch.dims, dtype=np.int32),
        nb=np.ascontiguousarray(batch.nb, dtype=np.int32),
        offset=np.ascontiguousarray(batch.offset, dtype=np.int64),
        fstride=np.ascontiguousarray(batch.fstride, dtype=np.int64),
        first=np.ascontiguousarray(first, dtype=np.int64),
    )
    T = BatchT(np=batch.np, ng=batch.g, dx=dx, **{k: v.ctypes.data for k, v in keep.items()})
    return T, keep


def _batch_lib():
    L = lib()
    if not getattr(L, "_batch_ready", False):
        dp = ctypes.POINTER(ctypes.c_double)
        L.or_batch_cycle.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(BatchT), dp, dp, dp,
                                     ctypes.POINTER(Particles), dp, dp, ctypes.c_void_p]
        L.or_batch_part.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(BatchT), ctypes.c_int32, ctypes.c_int32,
                                    dp, dp, ctypes.POINTER(Particles), dp, dp, ctypes.c_void_p]
        L.or_batch_fill_ghosts.argtypes = [ctypes.POINTER(BatchT), dp]
        L.or_batch_fold.argtypes = [ctypes.POINTER(BatchT), dp]
        L._batch_ready = True
    return L


def batch_fill_ghosts(batch, arena):
    """Every ghost cell := the cell of the neighbour patch it stands for."""
    T, keep = _batch_struct(batch, np.zeros(batch.np + 1, dtype=np.int64))
    _batch_lib().or_batch_fill_ghosts(ctypes.byref(T), _dp(arena))


def batch_fold(batch, arena):
    """Cross-patch ghost summation of a buffer arena, in place."""
    T, keep = _batch_struct(batch, np.zeros(batch.np + 1, dtype=np.int64))
    _batch_lib().or_batch_fold(ctypes.byref(T), _dp(arena))


def batch_cycle(params, batch, state, parts, first, dx=1.0, want_abs=False, want_eta=False):
    """One pass over a batch of patches (Steps 1-5).  Mutates the valid cells of
    ``state`` (an arena) and, for sinks, the particle mass and momentum.
    Returns dict(gathered, buf, absbuf, eta, counts)."""
    T, keep = _batch_struct(batch, first, dx)
    n = int(first[-1])
    assert len(parts["x"]) == n
    G = np.zeros((len(rows(params["kind"])), n))
    buf = batch.empty(0.0)
    absbuf = batch.empty(0.0) if want_abs else None
    eta = np.empty(batch.ncells_valid) if want_eta else None
    counts = np.zeros(2, dtype=np.int64)
    P = make_params(params)
    pp = make_particles(parts)
    st = _batch_lib().or_batch_cycle(ctypes.byref(P), ctypes.byref(T), _dp(state), _dp(buf), _dp(absbuf),
                                     ctypes.byref(pp), _dp(G), _dp(eta), counts.ctypes.data_as(ctypes.c_void_p))
    _check(st, "batch_cycle")
    return dict(gathered=G, buf=buf, absbuf=absbuf, eta=eta, counts=counts)


def batch_part(params, batch, owned, part, state, buf, parts, first, gathered, eta=None, dx=1.0):
    """One part of a pass over the first `owned` patches of a batch (part 0:
    Step 1; part 1: Steps 2-5), the other patches only read as neighbours;
    state, buf: arenas, mutated in place; gathered: [rows][total count].
    Returns the limiter counts of part 1."""
    T, keep = _batch_struct(batch, first, dx)
    counts = np.zeros(2, dtype=np.int64)
    P = make_params(params)
    pp = make_particles(parts)
    st = _batch_lib().or_batch_part(ctypes.byref(P), ctypes.byref(T), int(owned), int(part), _dp(state), _dp(buf),
                                    ctypes.byref(pp), _dp(gathered), _dp(eta), counts.ctypes.data_as(ctypes.c_void_p))
    _check(st, "batch_part")
    return counts
