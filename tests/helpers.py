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


def state_tolerance(params, U0, D, A, eta, tau=1e-12, chunk=1 << 20, dD=None, dlim=None):
    """Per cell and field bound on |U_new(GPU atomic) - U_new(oracle)| after
    Step 5 (tests/bounds.py): U0 the pre-update state, D, A and eta the
    oracle's summed buffer, sum of |dU| and eta, as (5, n), (5, n), (n,).
    Returns (tol, ambiguous)."""
    from bounds import U_ROUND, feedback_state_tolerance, sink_state_tolerance

    n = U0.shape[1]
    tol = np.empty((5, n))
    amb = np.zeros(n, dtype=bool)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        dd = None if dD is None else dD[:, a:b]
        if params["kind"] == "feedback":
            tol[:, a:b], amb[a:b] = feedback_state_tolerance(U0[:, a:b], D[:, a:b], A[:, a:b], tau, dd)
        elif params["kind"] == "sink":
            tol[:, a:b] = sink_state_tolerance(U0[:, a:b], D[:, a:b], A[:, a:b], eta[a:b], tau, dd,
                                               None if dlim is None else dlim[a:b])
        else:
            tol[:, a:b] = (tau * A[:, a:b] if dd is None else dd) + \
                4.0 * U_ROUND * (np.abs(U0[:, a:b]) + np.abs(D[:, a:b]))
    return tol, amb


def assert_state_within_bound(params, U0, D, A, eta, got, want, what="state after Step 5", tau=1e-12):
    """|got - want| within state_tolerance at every cell and field; returns
    the number of limiter-active cells and of ambiguous cells checked."""
    tol, amb = state_tolerance(params, U0, D, A, eta, tau)
    d = np.abs(got - want)
    bad = d > tol
    if np.any(bad):
        idx = np.argwhere(bad)[:5]
        f, c = idx[0]
        raise AssertionError(f"{what}: {np.count_nonzero(bad)} values exceed the derived bound, e.g. field {f} "
                             f"cell {c}: diff {d[f, c]:.3e} bound {tol[f, c]:.3e} (A {A[f, c]:.3e}, "
                             f"eta {eta[c]!r})")
    return int(np.count_nonzero(eta < 1.0)), int(np.count_nonzero(amb))


def sink_return_bound(params, box, state0, parts0, want, key):
    """Bound on |GPU - oracle| of sink quantity `key` after Step 4, per sink
    (tests/bounds.py: the removals differ only through eta)."""
    from bounds import sink_return_tolerance

    U = box.valid(state0).reshape(5, -1)
    vmax = 0.0
    for a in range(0, U.shape[1], 1 << 24):
        vmax = max(vmax, float(np.max(np.abs(U[1:4, a:a + (1 << 24)]) / U[0, a:a + (1 << 24)])))
    R = int(math.ceil(params["r_K"]))
    tm, tp = sink_return_tolerance(parts0["m"], want["m"], want[key], vmax, (2 * R + 1) ** 3)
    return tm if key == "m" else tp


FD_FIELDS = ("m", "e", "px", "py", "pz", "x", "y", "z")


def fd_step(f, one, Msnr):
    """Step of the finite difference of particle variable f: 1e-4 of the
    variable's scale (ejecta mass 1e-3), so that the quotient's rounding
    error (about eps * sum |terms| / h) stays small against 1e-8 of the
    derivative, while fourth-order differences keep the truncation error far
    below it.  Scales: m, E_sn themselves; a cell for positions; M_snr (the
    kernel's mass times a unit velocity) for the ejecta momentum, in which the
    deposit is exactly quadratic (v_COM linear, E_kin quadratic)."""
    if f == "m":
        return 1e-3 * abs(one["m"][0])
    if f == "e":
        return 1e-4 * abs(one["e"][0])
    if f in ("x", "y", "z"):
        return 1e-4
    return 1e-4 * Msnr


def fd_derivative(orc, params, box, state, one, Rv, f, Msnr):
    """d/df of L = sum_c R_c . Delta U^s_c over the particle's kernel cells
    (the oracle's deposition function of one particle, Eq. du), by the
    fourth-order central difference (4 D(h) - D(2h)) / 3 with the exact steps
    taken.  Returns (derivative, floor) with floor a bound on the quotient's
    own rounding error, or None when the kernel-cell set or the covered
    fractions change within +-2h (they carry no derivative)."""
    nx, ny, nz = box.n
    x0 = float(one[f][0])
    h = fd_step(f, one, Msnr)
    pts = [x0 - 2 * h, x0 - h, x0 + h, x0 + 2 * h]
    if f in ("x", "y", "z"):
        ks = [orc.kernel_of(params, box, *[(v if f == a else float(one[a][0])) for a in ("x", "y", "z")])
              for v in pts]
        if not all(np.array_equal(ks[0][0], k[0]) and np.array_equal(ks[0][1], k[1]) for k in ks):
            return None

    def L(val):
        o = {k: np.array(arr, dtype=np.float64, copy=True) for k, arr in one.items()}
        o[f][0] = val
        cells, dU = orc.deltas(params, box, state, o)
        terms = [float(Rv[c, kk % nz, jj % ny, ii % nx] * dU[q, c]) for q, (ii, jj, kk) in enumerate(cells)
                 for c in range(5)]
        return math.fsum(terms), math.fsum(abs(t) for t in terms)

    Ls = [L(v) for v in pts]
    h1, h2 = pts[2] - pts[1], pts[3] - pts[0]
    d1 = (Ls[2][0] - Ls[1][0]) / h1
    d2 = (Ls[3][0] - Ls[0][0]) / h2
    floor = 8.0 * EPS * max(t for _, t in Ls) / h1
    return (4.0 * d1 - d2) / 3.0, floor
