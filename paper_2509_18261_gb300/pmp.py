"""Python binding of the PMP C ABI (include/pmp.h).

Argument marshalling only: every step of the cycle runs in the CUDA kernels
of libpmp.so.  Meshes are float64 CUDA tensors of shape (5, field_stride);
particles are dicts of 1-D float64 CUDA tensors x, y, z, m, px, py, pz, e.
Each call enqueues on torch's current CUDA stream.

There is no CPU fallback: if libpmp.so is missing or no GPU is present, the
calls raise.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libpmp.so")

FEEDBACK, SINK, MASS = 0, 1, 2
ATOMIC, SORTED, ROUNDED = 0, 1, 2
KINDS = {"feedback": FEEDBACK, "sink": SINK, "mass": MASS}
MODES = {"atomic": ATOMIC, "sorted": SORTED, "rounded": ROUNDED}
STATUS = {
    0: "PMP_OK", 1: "PMP_ERR_ARG", 2: "PMP_ERR_GHOST_TOO_THIN", 3: "PMP_ERR_PARTICLE_OUTSIDE",
    4: "PMP_ERR_NONFINITE", 5: "PMP_ERR_TIMEOUT", 6: "PMP_ERR_WORKSPACE", 7: "PMP_ERR_CUDA",
}
EXPORTS = [
    "pmp_create", "pmp_destroy", "pmp_set_stream", "pmp_set_rounding_margin", "pmp_gathered_rows", "pmp_workspace_size", "pmp_zero_buffer",
    "pmp_gather", "pmp_deposit", "pmp_gather_deposit", "pmp_fold_ghosts", "pmp_apply_limited", "pmp_backward", "pmp_get_error",
    "pmp_limiter_counts", "pmp_timing_enable", "pmp_timing_read", "pmp_deposit_noalloc",
    "pmp_create_sinks_workspace_size", "pmp_create_sinks", "pmp_apply_extra",
    "pmp_batch_create", "pmp_batch_set_particles", "pmp_batch_set_strategy", "pmp_batch_strategies",
    "pmp_batch_autotune", "pmp_cycle_batched", "pmp_batch_info", "pmp_batch_hold_barriers", "pmp_batch_destroy",
    "pmp_probe_threads", "pmp_probe_chains", "pmp_probe_fp64", "pmp_probe_atomic", "pmp_exact_math",
    "pmp_partition_sfc", "pmp_plan_create", "pmp_plan_local", "pmp_plan_regions", "pmp_plan_destroy",
    "pmp_batch_create_partial", "pmp_cycle_batched_part", "pmp_batch_set_regions", "pmp_batch_pack",
    "pmp_batch_unpack",
]
PART_ALL, PART_DEPOSIT, PART_FINISH = 0, 1, 2
XCH_STATE, XCH_GHOST, XCH_FOLDED = 0, 1, 2
PERSISTENT, PER_PATCH, GRAPH = 0, 1, 2
LAUNCHES = {"persistent": PERSISTENT, "per_patch": PER_PATCH, "graph": GRAPH}
OWNER_CUBE, OWNER_ROWS, STRAT_ATOMIC = 0, 1, 2
STRATEGIES = {"owner_cube": OWNER_CUBE, "owner_rows": OWNER_ROWS, "atomic": STRAT_ATOMIC}
BATCH_BINS = 20


class PMPError(RuntimeError):
    def __init__(self, what, code):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


class _Params(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("subsample", ctypes.c_int32),
        ("r_K", ctypes.c_double), ("dt", ctypes.c_double), ("G", ctypes.c_double),
        ("gamma", ctypes.c_double), ("lambda_bh", ctypes.c_double), ("J", ctypes.c_double),
        ("cap", ctypes.c_double), ("rho_min", ctypes.c_double), ("A_sf", ctypes.c_double),
        ("A_p", ctypes.c_double), ("mu_H", ctypes.c_double), ("RM_ej", ctypes.c_double),
        ("RM_st", ctypes.c_double), ("eps_K", ctypes.c_double),
    ]


class _Mesh(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 3), ("ng", ctypes.c_int32), ("periodic", ctypes.c_int32 * 3),
        ("reserved", ctypes.c_int32), ("dx", ctypes.c_double), ("field_stride", ctypes.c_int64),
        ("data", ctypes.c_void_p),
    ]


class _KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("ms", ctypes.c_double)]


class _Patch(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("neighbour", ctypes.c_int32 * 26), ("offset", ctypes.c_int64),
                ("field_stride", ctypes.c_int64)]


class _Region(ctypes.Structure):
    _fields_ = [("peer", ctypes.c_int32), ("patch", ctypes.c_int32), ("lo", ctypes.c_int32 * 3),
                ("hi", ctypes.c_int32 * 3), ("offset", ctypes.c_int64)]


class _Particles(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_int64), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
        ("m", ctypes.c_void_p), ("px", ctypes.c_void_p), ("py", ctypes.c_void_p), ("pz", ctypes.c_void_p),
        ("e", ctypes.c_void_p),
    ]


_lib = None


def load():
    """Load libpmp.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libpmp.so not found at {LIB_PATH}: build it first (__graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    P, M, Pa = ctypes.POINTER(_Params), ctypes.POINTER(_Mesh), ctypes.POINTER(_Particles)
    sig = {
        "pmp_create": ([ctypes.POINTER(vp), P, vp], i32),
        "pmp_destroy": ([vp], None),
        "pmp_set_stream": ([vp, vp], i32),
        "pmp_set_rounding_margin": ([vp, i32], i32),
        "pmp_gathered_rows": ([i32], i32),
        "pmp_workspace_size": ([vp, M, i64, i32, ctypes.POINTER(ctypes.c_size_t)], i32),
        "pmp_zero_buffer": ([vp, M], i32),
        "pmp_gather": ([vp, M, Pa, vp, i32, vp, ctypes.c_size_t], i32),
        "pmp_deposit": ([vp, M, Pa, vp, M, i32, vp, ctypes.c_size_t], i32),
        "pmp_gather_deposit": ([vp, M, Pa, vp, M, i32, vp, ctypes.c_size_t], i32),
        "pmp_fold_ghosts": ([vp, M], i32),
        "pmp_apply_limited": ([vp, M, M, Pa, vp, vp, vp, ctypes.c_size_t], i32),
        "pmp_backward": ([vp, M, M, Pa, vp, vp, vp, vp, ctypes.c_size_t], i32),
        "pmp_get_error": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i64)], i32),
        "pmp_limiter_counts": ([vp, ctypes.POINTER(i64)], i32),
        "pmp_timing_enable": ([vp, i32], i32),
        "pmp_timing_read": ([vp, ctypes.POINTER(_KernelTime), i32, ctypes.POINTER(i32)], i32),
        "pmp_deposit_noalloc": ([P, M, Pa, vp, M, vp], i32),
        "pmp_create_sinks_workspace_size": ([vp, M, ctypes.POINTER(ctypes.c_size_t)], i32),
        "pmp_apply_extra": ([vp, M, M, vp, i32, i64], i32),
        "pmp_create_sinks": ([vp, M, M, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_size_t], i32),
        "pmp_batch_create": ([vp, ctypes.POINTER(_Patch), i32, i32, ctypes.c_double, i64, ctypes.POINTER(vp)], i32),
        "pmp_batch_set_particles": ([vp, ctypes.POINTER(i64)], i32),
        "pmp_batch_set_strategy": ([vp, i32], i32),
        "pmp_batch_strategies": ([vp, ctypes.POINTER(i32)], i32),
        "pmp_batch_autotune": ([vp, vp, vp, Pa, vp, i32, i32, ctypes.POINTER(i32)], i32),
        "pmp_cycle_batched": ([vp, vp, vp, Pa, vp, vp, i32], i32),
        "pmp_batch_info": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i64)], i32),
        "pmp_batch_hold_barriers": ([vp, i32], i32),
        "pmp_batch_destroy": ([vp], None),
        "pmp_probe_threads": ([], i32),
        "pmp_probe_chains": ([], i32),
        "pmp_probe_fp64": ([vp, i32, i32, vp], i32),
        "pmp_probe_atomic": ([vp, i64, i64, i32, vp], i32),
        "pmp_exact_math": ([vp, vp, i64, vp, vp, vp], i32),
        "pmp_partition_sfc": ([i32, ctypes.POINTER(i32), ctypes.POINTER(i64), i32, ctypes.POINTER(i32)], i32),
        "pmp_plan_create": ([ctypes.POINTER(_Patch), i32, i32, ctypes.POINTER(i32), i32, i32, ctypes.POINTER(vp)],
                            i32),
        "pmp_plan_local": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(_Patch),
                            ctypes.POINTER(i32), ctypes.POINTER(i64)], i32),
        "pmp_plan_regions": ([vp, i32, i32, ctypes.POINTER(_Region), i32, ctypes.POINTER(i32)], i32),
        "pmp_plan_destroy": ([vp], None),
        "pmp_batch_create_partial": ([vp, ctypes.POINTER(_Patch), i32, i32, i32, ctypes.c_double, i64,
                                      ctypes.POINTER(vp)], i32),
        "pmp_cycle_batched_part": ([vp, vp, vp, Pa, vp, vp, i32, i32], i32),
        "pmp_batch_set_regions": ([vp, i32, ctypes.POINTER(_Region), i32], i32),
        "pmp_batch_pack": ([vp, i32, vp, vp, i32], i32),
        "pmp_batch_unpack": ([vp, i32, vp, vp], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(what, code):
    if code != 0:
        raise PMPError(what, code)


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError("expected a float64 CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


class Mesh:
    """A (5, field_stride) float64 CUDA tensor with its box geometry."""

    def __init__(self, data, n, ng, periodic=(1, 1, 1), dx=1.0):
        if data.dim() != 2 or data.shape[0] != 5:
            raise ValueError("mesh data must have shape (5, field_stride)")
        self.data, self.n, self.ng = data, tuple(int(v) for v in n), int(ng)
        self.periodic, self.dx = tuple(int(v) for v in periodic), float(dx)

    def c(self):
        return _Mesh(n=(ctypes.c_int32 * 3)(*self.n), ng=self.ng, periodic=(ctypes.c_int32 * 3)(*self.periodic),
                     reserved=0, dx=self.dx, field_stride=self.data.shape[1], data=_ptr(self.data))


def _parts(p):
    if p is None:
        return None
    n = int(p["x"].numel())
    return _Particles(count=n, x=_ptr(p["x"]), y=_ptr(p["y"]), z=_ptr(p["z"]), m=_ptr(p["m"]), px=_ptr(p["px"]),
                      py=_ptr(p["py"]), pz=_ptr(p["pz"]), e=_ptr(p.get("e")))


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Context:
    """An opaque pmp_ctx for one interaction kind (pmp_create / pmp_destroy)."""

    def __init__(self, params):
        L = load()
        self.params = dict(params)
        self.kind = KINDS[params["kind"]]
        cp = _Params(kind=self.kind, subsample=int(params["subsample"]), r_K=params["r_K"], dt=params["dt"],
                     G=params["G"], gamma=params["gamma"], lambda_bh=params["lambda_bh"], J=params["J"],
                     cap=params["cap"], rho_min=params["rho_min"], A_sf=params["A_sf"], A_p=params["A_p"],
                     mu_H=params["mu_H"], RM_ej=params["RM_ej"], RM_st=params["RM_st"], eps_K=params["eps_K"])
        h = ctypes.c_void_p()
        _check("pmp_create", L.pmp_create(ctypes.byref(h), ctypes.byref(cp), _stream()))
        self.h = h

    def _sync_stream(self):
        _check("pmp_set_stream", load().pmp_set_stream(self.h, _stream()))

    def close(self):
        if getattr(self, "h", None):
            load().pmp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pmp_create(params):
    return Context(params)


def pmp_apply_extra(ctx, state, buffer, extra):
    """Auxiliary fields at fixed specific value under accretion: ``extra`` is a
    (n_extra, field_stride) float64 CUDA tensor laid out like the state."""
    ctx._sync_stream()
    n = int(extra.shape[0]) if extra.dim() == 2 else 1
    stride = int(extra.shape[-1])
    _check("pmp_apply_extra", load().pmp_apply_extra(ctx.h, ctypes.byref(state.c()), ctypes.byref(buffer.c()),
                                                     _ptr(extra), n, stride))


def pmp_create_sinks_workspace_size(ctx, state):
    out = ctypes.c_size_t()
    _check("pmp_create_sinks_workspace_size",
           load().pmp_create_sinks_workspace_size(ctx.h, ctypes.byref(state.c()), ctypes.byref(out)))
    return out.value


def pmp_create_sinks(ctx, state, buffer, out, count, workspace):
    """Sink creation (Sec. 3.1.2): ``out`` is a dict of device arrays x, y, z,
    m, px, py, pz (their length is the capacity); ``count`` a device int64
    tensor of one element receiving the number of qualifying cells."""
    ctx._sync_stream()
    cap = int(out["x"].numel())
    ws, wsb = _ws(workspace)
    args = [_ptr(out[k]) for k in ("x", "y", "z", "m", "px", "py", "pz")]
    if not (isinstance(count, torch.Tensor) and count.is_cuda and count.dtype == torch.int64 and count.numel() >= 1):
        raise TypeError("count must be a CUDA int64 tensor")
    _check("pmp_create_sinks", load().pmp_create_sinks(ctx.h, ctypes.byref(state.c()), ctypes.byref(buffer.c()),
                                                       cap, *args, ctypes.c_void_p(count.data_ptr()), ws, wsb))


def pmp_set_rounding_margin(ctx, M):
    """Safety margin M of the ROUNDED deposit (App. A.1)."""
    _check("pmp_set_rounding_margin", load().pmp_set_rounding_margin(ctx.h, int(M)))


def pmp_gathered_rows(kind):
    return load().pmp_gathered_rows(KINDS.get(kind, kind))


def pmp_workspace_size(ctx, buffer, n_particles, mode):
    out = ctypes.c_size_t()
    _check("pmp_workspace_size",
           load().pmp_workspace_size(ctx.h, ctypes.byref(buffer.c()), int(n_particles), MODES.get(mode, mode),
                                     ctypes.byref(out)))
    return out.value


def pmp_zero_buffer(ctx, buffer):
    ctx._sync_stream()
    _check("pmp_zero_buffer", load().pmp_zero_buffer(ctx.h, ctypes.byref(buffer.c())))


def _ws(workspace):
    if workspace is None:
        return None, 0
    if not workspace.is_cuda or not workspace.is_contiguous():
        raise ValueError("workspace must be a contiguous CUDA tensor")
    return ctypes.c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size()


def pmp_gather(ctx, state, parts, gathered, mode="atomic", workspace=None):
    ctx._sync_stream()
    pp = _parts(parts)
    ws, wsb = _ws(workspace)
    _check("pmp_gather", load().pmp_gather(ctx.h, ctypes.byref(state.c()), ctypes.byref(pp), _ptr(gathered),
                                           MODES.get(mode, mode), ws, wsb))


def pmp_deposit(ctx, state, parts, gathered, buffer, mode="atomic", workspace=None):
    ctx._sync_stream()
    pp = _parts(parts)
    ws, wsb = _ws(workspace)
    _check("pmp_deposit", load().pmp_deposit(ctx.h, ctypes.byref(state.c()), ctypes.byref(pp), _ptr(gathered),
                                             ctypes.byref(buffer.c()), MODES.get(mode, mode), ws, wsb))


def pmp_gather_deposit(ctx, state, parts, gathered, buffer, mode="atomic", workspace=None):
    ctx._sync_stream()
    pp = _parts(parts)
    ws, wsb = _ws(workspace)
    _check("pmp_gather_deposit",
           load().pmp_gather_deposit(ctx.h, ctypes.byref(state.c()), ctypes.byref(pp), _ptr(gathered),
                                     ctypes.byref(buffer.c()), MODES.get(mode, mode), ws, wsb))


def pmp_fold_ghosts(ctx, buffer):
    ctx._sync_stream()
    _check("pmp_fold_ghosts", load().pmp_fold_ghosts(ctx.h, ctypes.byref(buffer.c())))


def pmp_apply_limited(ctx, state, buffer, parts=None, gathered=None, eta_out=None, workspace=None):
    ctx._sync_stream()
    pp = _parts(parts)
    ws, wsb = _ws(workspace)
    _check("pmp_apply_limited",
           load().pmp_apply_limited(ctx.h, ctypes.byref(state.c()), ctypes.byref(buffer.c()),
                                    ctypes.byref(pp) if pp is not None else None, _ptr(gathered), _ptr(eta_out),
                                    ws, wsb))


def pmp_backward(ctx, state_in, buffer, parts, gathered, gU, g_out, workspace=None):
    ctx._sync_stream()
    pp = _parts(parts)
    ws, wsb = _ws(workspace)
    _check("pmp_backward", load().pmp_backward(ctx.h, ctypes.byref(state_in.c()), ctypes.byref(buffer.c()),
                                               ctypes.byref(pp), _ptr(gathered), _ptr(gU), _ptr(g_out), ws, wsb))


def pmp_get_error(ctx):
    code, idx = ctypes.c_int32(), ctypes.c_int64()
    ctx._sync_stream()
    _check("pmp_get_error", load().pmp_get_error(ctx.h, ctypes.byref(code), ctypes.byref(idx)))
    return code.value, idx.value


def pmp_limiter_counts(ctx):
    c = (ctypes.c_int64 * 2)()
    ctx._sync_stream()
    _check("pmp_limiter_counts", load().pmp_limiter_counts(ctx.h, c))
    return c[0], c[1]


def _params_struct(params):
    return _Params(kind=KINDS[params["kind"]], subsample=int(params["subsample"]), r_K=params["r_K"],
                   dt=params["dt"], G=params["G"], gamma=params["gamma"], lambda_bh=params["lambda_bh"],
                   J=params["J"], cap=params["cap"], rho_min=params["rho_min"], A_sf=params["A_sf"],
                   A_p=params["A_p"], mu_H=params["mu_H"], RM_ej=params["RM_ej"], RM_st=params["RM_st"],
                   eps_K=params["eps_K"])


def pmp_deposit_noalloc(params, state, parts, gathered, buffer):
    """Supernova gather + atomic deposit with the library's fixed scratch (no
    device allocation by the library; see include/pmp.h)."""
    cp = _params_struct(params)
    pp = _parts(parts)
    _check("pmp_deposit_noalloc", load().pmp_deposit_noalloc(ctypes.byref(cp), ctypes.byref(state.c()),
                                                             ctypes.byref(pp), _ptr(gathered),
                                                             ctypes.byref(buffer.c()), _stream()))


def pmp_probe_threads():
    return load().pmp_probe_threads()


def pmp_probe_chains():
    return load().pmp_probe_chains()


def pmp_probe_fp64(out, blocks, iters):
    """Enqueues the FP64 fused multiply-add probe on the current stream."""
    _check("pmp_probe_fp64", load().pmp_probe_fp64(_ptr(out), blocks, iters, _stream()))


def pmp_probe_atomic(target, n_adds, blocks):
    """Enqueues n_adds FP64 atomicAdd over the doubles of `target`."""
    _check("pmp_probe_atomic", load().pmp_probe_atomic(_ptr(target), target.numel(), n_adds, blocks, _stream()))


def pmp_exact_math(a, b, quot, root):
    """quot = a / b and root = sqrt(a), element-wise, by the library's integer
    forms (device tensors of float64, same length)."""
    n = a.numel()
    if not (b.numel() == quot.numel() == root.numel() == n):
        raise ValueError("pmp_exact_math: arrays of different lengths")
    _check("pmp_exact_math", load().pmp_exact_math(_ptr(a), _ptr(b), n, _ptr(quot), _ptr(root), _stream()))


def pmp_timing_enable(ctx, on=True):
    _check("pmp_timing_enable", load().pmp_timing_enable(ctx.h, 1 if on else 0))


def pmp_timing_read(ctx):
    """{kernel name: (launches, total ms)} since the last read (synchronises)."""
    buf = (_KernelTime * 64)()
    n = ctypes.c_int32()
    ctx._sync_stream()
    _check("pmp_timing_read", load().pmp_timing_read(ctx.h, buf, 64, ctypes.byref(n)))
    return {buf[i].name.decode(): (buf[i].launches, buf[i].ms) for i in range(min(n.value, 64))}


class BatchHandle:
    """An opaque pmp_batch (pmp_batch_create / pmp_batch_destroy).

    ``dims`` (np, 3), ``nb`` (np, 26), ``offset`` and ``field_stride`` (np)
    describe the patches (host arrays); ``ctx`` fixes the interaction kind."""

    def __init__(self, ctx, dims, nb, offset, field_stride, ng, arena_len, dx=1.0, n_owned=None):
        L = load()
        n = len(dims)
        arr = _patch_array(dims, nb, offset, field_stride)
        ctx._sync_stream()
        h = ctypes.c_void_p()
        if n_owned is None:
            _check("pmp_batch_create", L.pmp_batch_create(ctx.h, arr, n, int(ng), float(dx), int(arena_len),
                                                          ctypes.byref(h)))
        else:
            _check("pmp_batch_create_partial", L.pmp_batch_create_partial(ctx.h, arr, n, int(n_owned), int(ng),
                                                                          float(dx), int(arena_len),
                                                                          ctypes.byref(h)))
        self.h, self.ctx, self.np = h, ctx, n

    def close(self):
        if getattr(self, "h", None):
            load().pmp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _patch_array(dims, nb, offset=None, field_stride=None):
    n = len(dims)
    arr = (_Patch * n)()
    for p in range(n):
        arr[p].n = (ctypes.c_int32 * 3)(*[int(v) for v in dims[p]])
        arr[p].neighbour = (ctypes.c_int32 * 26)(*[int(v) for v in nb[p]])
        arr[p].offset = int(offset[p]) if offset is not None else 0
        arr[p].field_stride = int(field_stride[p]) if field_stride is not None else 0
    return arr


def pmp_batch_create(ctx, dims, nb, offset, field_stride, ng, arena_len, dx=1.0):
    return BatchHandle(ctx, dims, nb, offset, field_stride, ng, arena_len, dx)


def pmp_batch_create_partial(ctx, dims, nb, offset, field_stride, n_owned, ng, arena_len, dx=1.0):
    return BatchHandle(ctx, dims, nb, offset, field_stride, ng, arena_len, dx, n_owned=n_owned)


def pmp_cycle_batched_part(batch, state, buffer, parts, gathered, eta_out=None, launch="persistent", part=PART_ALL):
    pp = _parts(parts)
    batch.ctx._sync_stream()
    _check("pmp_cycle_batched_part", load().pmp_cycle_batched_part(batch.h, _ptr(state), _ptr(buffer),
                                                                   ctypes.byref(pp), _ptr(gathered), _ptr(eta_out),
                                                                   LAUNCHES.get(launch, launch), int(part)))


def _region_array(regions):
    arr = (_Region * max(len(regions), 1))()
    for i, r in enumerate(regions):
        arr[i].peer, arr[i].patch = int(r["peer"]), int(r["patch"])
        arr[i].lo = (ctypes.c_int32 * 3)(*[int(v) for v in r["lo"]])
        arr[i].hi = (ctypes.c_int32 * 3)(*[int(v) for v in r["hi"]])
        arr[i].offset = int(r["offset"])
    return arr


def pmp_batch_set_regions(batch, slot, regions):
    batch.ctx._sync_stream()
    _check("pmp_batch_set_regions", load().pmp_batch_set_regions(batch.h, int(slot), _region_array(regions),
                                                                 len(regions)))


def pmp_batch_pack(batch, slot, arena, msg, folded=False):
    batch.ctx._sync_stream()
    _check("pmp_batch_pack", load().pmp_batch_pack(batch.h, int(slot), _ptr(arena), _ptr(msg), 1 if folded else 0))


def pmp_batch_unpack(batch, slot, msg, arena):
    batch.ctx._sync_stream()
    _check("pmp_batch_unpack", load().pmp_batch_unpack(batch.h, int(slot), _ptr(msg), _ptr(arena)))


# host-only plan calls (no GPU needed)

def pmp_partition_sfc(pos, cost, n_ranks):
    """rank_of per patch (list) from super-grid positions (n, 3) and costs."""
    n = len(pos)
    P = (ctypes.c_int32 * (3 * n))(*[int(v) for row in pos for v in row])
    C = (ctypes.c_int64 * n)(*[int(v) for v in cost])
    out = (ctypes.c_int32 * n)()
    _check("pmp_partition_sfc", load().pmp_partition_sfc(n, P, C, int(n_ranks), out))
    return list(out)


class PlanHandle:
    """An opaque pmp_plan (pmp_plan_create / pmp_plan_destroy)."""

    def __init__(self, dims, nb, ng, rank_of, n_ranks, rank):
        n = len(dims)
        arr = _patch_array(dims, nb)
        ro = (ctypes.c_int32 * n)(*[int(v) for v in rank_of])
        h = ctypes.c_void_p()
        _check("pmp_plan_create", load().pmp_plan_create(arr, n, int(ng), ro, int(n_ranks), int(rank),
                                                         ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().pmp_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pmp_plan_create(dims, nb, ng, rank_of, n_ranks, rank):
    return PlanHandle(dims, nb, ng, rank_of, n_ranks, rank)


def pmp_plan_local(plan):
    """dict(n_owned, dims (n, 3), nb (n, 26), offset, field_stride, global_id, arena_len)."""
    L = load()
    no, nl, al = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check("pmp_plan_local", L.pmp_plan_local(plan.h, ctypes.byref(no), ctypes.byref(nl), None, None,
                                              ctypes.byref(al)))
    arr = (_Patch * nl.value)()
    gid = (ctypes.c_int32 * nl.value)()
    _check("pmp_plan_local", L.pmp_plan_local(plan.h, None, None, arr, gid, None))
    return dict(n_owned=no.value, dims=[tuple(arr[i].n) for i in range(nl.value)],
                nb=[tuple(arr[i].neighbour) for i in range(nl.value)],
                offset=[arr[i].offset for i in range(nl.value)],
                field_stride=[arr[i].field_stride for i in range(nl.value)],
                global_id=list(gid), arena_len=al.value)


def pmp_plan_regions(plan, kind, send):
    """List of dict(peer, patch, lo, hi, offset)."""
    L = load()
    n = ctypes.c_int32()
    _check("pmp_plan_regions", L.pmp_plan_regions(plan.h, int(kind), int(send), None, 0, ctypes.byref(n)))
    arr = (_Region * max(n.value, 1))()
    _check("pmp_plan_regions", L.pmp_plan_regions(plan.h, int(kind), int(send), arr, n.value, ctypes.byref(n)))
    return [dict(peer=arr[i].peer, patch=arr[i].patch, lo=tuple(arr[i].lo), hi=tuple(arr[i].hi),
                 offset=arr[i].offset) for i in range(n.value)]


def pmp_batch_set_particles(batch, first):
    arr = (ctypes.c_int64 * len(first))(*[int(v) for v in first])
    batch.ctx._sync_stream()
    _check("pmp_batch_set_particles", load().pmp_batch_set_particles(batch.h, arr))


def pmp_batch_set_strategy(batch, strategy):
    batch.ctx._sync_stream()
    _check("pmp_batch_set_strategy", load().pmp_batch_set_strategy(batch.h, STRATEGIES.get(strategy, strategy)))


def pmp_batch_strategies(batch):
    out = (ctypes.c_int32 * batch.np)()
    _check("pmp_batch_strategies", load().pmp_batch_strategies(batch.h, out))
    return list(out)


def pmp_batch_autotune(batch, state, buffer, parts, gathered, deterministic=False, reps=3):
    """Returns the chosen strategy per bin (-1: empty bin)."""
    pp = _parts(parts)
    out = (ctypes.c_int32 * BATCH_BINS)()
    batch.ctx._sync_stream()
    _check("pmp_batch_autotune", load().pmp_batch_autotune(batch.h, _ptr(state), _ptr(buffer), ctypes.byref(pp),
                                                           _ptr(gathered), 1 if deterministic else 0, int(reps),
                                                           out))
    return list(out)


def pmp_cycle_batched(batch, state, buffer, parts, gathered, eta_out=None, launch="persistent"):
    pp = _parts(parts)
    batch.ctx._sync_stream()
    _check("pmp_cycle_batched", load().pmp_cycle_batched(batch.h, _ptr(state), _ptr(buffer), ctypes.byref(pp),
                                                         _ptr(gathered), _ptr(eta_out), LAUNCHES.get(launch, launch)))


def pmp_batch_hold_barriers(batch, arrivals):
    _check("pmp_batch_hold_barriers", load().pmp_batch_hold_barriers(batch.h, int(arrivals)))


def pmp_batch_info(batch):
    g = ctypes.c_int32()
    it = (ctypes.c_int64 * 3)()
    _check("pmp_batch_info", load().pmp_batch_info(batch.h, ctypes.byref(g), it))
    return g.value, tuple(it)


# ---------------------------------------------------------------------------
# conveniences built only from the calls above
# ---------------------------------------------------------------------------

def to_device(arr, device="cuda"):
    return torch.from_numpy(arr).to(device)


def parts_to_device(p, device="cuda"):
    return {k: torch.from_numpy(v).to(device) for k, v in p.items()}


class Pass:
    """One PMP pass (zero, gather, deposit, fold, limited apply) of one kind
    on one box, with its buffers allocated once.  `fused`: gather and deposit
    through pmp_gather_deposit (else pmp_gather, then pmp_deposit)."""

    def __init__(self, params, box, state, parts, mode="atomic", dx=1.0, periodic=(1, 1, 1), want_eta=False,
                 fused=True):
        self.ctx = Context(params)
        self.box, self.mode, self.fused = box, mode, fused
        dev = state.device
        self.state = Mesh(state, box.n, box.g, periodic, dx)
        self.buffer = Mesh(torch.empty((5, box.field_stride), dtype=torch.float64, device=dev), box.n, box.g,
                           periodic, dx)
        self.parts = parts
        n = int(parts["x"].numel()) if parts is not None else 0
        self.gathered = torch.empty((pmp_gathered_rows(params["kind"]), max(n, 1)), dtype=torch.float64, device=dev)
        self.eta = torch.empty(box.ncells_valid, dtype=torch.float64, device=dev) if want_eta else None
        nbytes = pmp_workspace_size(self.ctx, self.buffer, n, mode)
        self.workspace = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)

    def gathered_view(self):
        n = int(self.parts["x"].numel())
        return self.gathered[:, :n]

    def run(self, stop_after=None):
        c = self.ctx
        has = self.parts is not None and self.parts["x"].numel() > 0
        pmp_zero_buffer(c, self.buffer)
        if has and self.fused:
            pmp_gather_deposit(c, self.state, self.parts, self.gathered, self.buffer, self.mode, self.workspace)
        else:
            pmp_gather(c, self.state, self.parts if has else _EMPTY(self.state.data.device), self.gathered,
                       self.mode, self.workspace)
            if has:
                pmp_deposit(c, self.state, self.parts, self.gathered, self.buffer, self.mode, self.workspace)
        if stop_after == "deposit":
            return
        pmp_fold_ghosts(c, self.buffer)
        if stop_after == "fold":
            return
        pmp_apply_limited(c, self.state, self.buffer, self.parts if has else None, self.gathered if has else None,
                          self.eta, self.workspace)


def _EMPTY(device):
    z = torch.zeros(1, dtype=torch.float64, device=device)
    return {k: z[:0] for k in ("x", "y", "z", "m", "px", "py", "pz", "e")}


class BatchPass:
    """One pass of one kind over a synthetic.Batch of patches: state and
    buffer arenas, particles (patch after patch), gathered rows, the batch
    handle with its particle ranges set."""

    def __init__(self, params, batch, state, parts, first, dx=1.0, want_eta=False):
        self.ctx = Context(params)
        dev = state.device
        self.batch = batch
        self.state = state
        self.buffer = torch.zeros(batch.arena_len, dtype=torch.float64, device=dev)
        self.parts = parts
        n = int(parts["x"].numel())
        self.n = n
        self.gathered = torch.zeros((pmp_gathered_rows(params["kind"]), max(n, 1)), dtype=torch.float64, device=dev)
        self.eta = torch.empty(batch.ncells_valid, dtype=torch.float64, device=dev) if want_eta else None
        self.h = BatchHandle(self.ctx, batch.dims, batch.nb, batch.offset, batch.fstride, batch.g, batch.arena_len,
                             dx)
        pmp_batch_set_particles(self.h, first)

    def gathered_view(self):
        return self.gathered[:, : self.n]

    def run(self, launch="persistent"):
        pmp_cycle_batched(self.h, self.state, self.buffer, self.parts, self.gathered, self.eta, launch)

    def close(self):
        self.h.close()
        self.ctx.close()
