"""Shared helpers of the GPU tests: run one pass on the GPU through the C ABI
binding and the same pass in the oracle, on the same seeded inputs."""
import math

import numpy as np

from paper_2509_18261_gb300 import synthetic as syn

EPS = 2.0 ** -52


def cuda_ok():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


def gpu_pass(params, box, state_np, parts_np, mode="atomic", periodic=(1, 1, 1), dx=1.0, stop_after=None):
    """Runs one pass on the GPU.  Returns dict of numpy arrays: state (after),
    buf (after the requested stage), gathered, eta, parts (after), counts,
    error.  Mode "atomic-split": the atomic mode through pmp_gather and
    pmp_deposit (else gather and deposit go through pmp_gather_deposit)."""
    import torch

    from paper_2509_18261_gb300 import pmp

    dev = "cuda"
    st = torch.from_numpy(state_np.copy()).to(dev)
    parts = pmp.parts_to_device(parts_np, dev) if parts_np is not None else None
    fused = mode != "atomic-split"
    mode = "atomic" if mode == "atomic-split" else mode
    ps = pmp.Pass(params, box, st, parts, mode=mode, dx=dx, periodic=periodic, want_eta=True, fused=fused)
    ps.run(stop_after=stop_after)
    torch.cuda.synchronize()
    out = dict(
        state=st.cpu().numpy(),
        buf=ps.buffer.data.cpu().numpy(),
        eta=ps.eta.cpu().numpy(),
        error=pmp.pmp_get_error(ps.ctx),
        counts=pmp.pmp_limiter_counts(ps.ctx),
    )
    if parts is not None and parts_np["x"].size:
        out["gathered"] = ps.gathered_view().cpu().numpy()
        out["parts"] = {k: v.cpu().numpy() for k, v in parts.items()}
    ps.ctx.close()
    return out


def oracle_pass(orc, params, box, state_np, parts_np, periodic=(1, 1, 1), dx=1.0):
    st = state_np.copy()
    parts = {k: v.copy() for k, v in parts_np.items()} if parts_np is not None else None
    if parts is None or parts["x"].size == 0:
        buf = box.empty(0.0)
        eta, counts = orc.apply(params, box, st, buf, dx, periodic, want_eta=True)
        return dict(state=st, buf=buf, pre_fold=buf.copy(), absbuf=box.empty(0.0), eta=eta, counts=counts,
                    parts=parts)
    r = orc.cycle(params, box, st, parts, dx=dx, periodic=periodic, want_abs=True, want_eta=True)
    r["state"] = st
    r["parts"] = parts
    return r


def assert_bits_equal(a, b, what):
    a = np.asarray(a)
    b = np.asarray(b)
    assert a.shape == b.shape, what
    same = (a.view(np.uint64) == b.view(np.uint64)) | (np.isnan(a) & np.isnan(b))
    if not np.all(same):
        idx = np.argwhere(~same)[:5]
        raise AssertionError(f"{what}: {np.count_nonzero(~same)} values differ, e.g. at {idx.tolist()}: "
                             f"{a[tuple(idx[0])]!r} vs {b[tuple(idx[0])]!r}")


def assert_within_abs(gpu, ora, absum, what, rel=1e-12):
    """|gpu - oracle| <= rel * A_c per cell and field (A_c = sum of |dU|)."""
    d = np.abs(gpu - ora)
    bad = d > rel * absum
    if np.any(bad):
        idx = np.argwhere(bad)[:5]
        raise AssertionError(f"{what}: {np.count_nonzero(bad)} cells exceed {rel} * A_c, e.g. {idx.tolist()} "
                             f"diff {d[tuple(idx[0])]:.3e} A {absum[tuple(idx[0])]:.3e}")


def valid_flat(box, arr):
    return box.valid(arr).reshape(5, -1)
