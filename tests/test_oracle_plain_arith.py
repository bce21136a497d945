"""The oracle's evaluation-order readings change only rounding.

The oracle fuses a product into the sum it feeds in a few places (fma: the
supernova gather sums, the sum of the sink kernel weights, the momentum and
energy rows of Eq. du, the Step-4 sums) and evaluates every quotient by rho in
the sink formulas as a product with the cell's one reciprocal 1/rho.  In
real arithmetic both are the printed formulas.  This test builds a second
copy of the oracle in which every fma(a, b, c) is the separately rounded
a * b + c and every product with that reciprocal is the quotient by rho
itself, and checks that

- every pin of the oracle passes on the copy too;
- on the 32^3 workload (supernovae, then sinks), boxes with edge geometry and
  a clustered box, the copy agrees with the oracle to within rounding: the
  gathered rows to a few units of the last place, the buffer to a few
  eps * A_c per cell and field (A_c = sum_s |Delta U^s_c|), the state after
  Step 5 and the sinks after Step 4 within the bounds that such a buffer
  difference implies through the limiters (tests/bounds.py).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from helpers import state_tolerance

from paper_2509_18261_gb300 import synthetic as syn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pmp_oracle.c")
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_create.py", "tests/test_oracle_extra.py",
        "tests/test_oracle_mass.py", "tests/test_oracle_batch.py", "tests/test_oracle_repro.py"]
EPS = 2.0 ** -52

# (original text, separately rounded form); each original occurs once
PLAIN = [
    ("#include <string.h>\n", "#include <string.h>\n#undef fma\n#define fma(a, b, c) ((a) * (b) + (c))\n"),
    ("    double eint = U[4] - ke2 * (0.5 * inv);", "    double eint = U[4] - ke2 / (2.0 * U[0]);"),
    ("    double cs2 = (gg * eint) * inv;", "    double cs2 = (gg * eint) / U[0];"),
    ("    for (int k = 0; k < 3; k++) dU[1 + k] = -(a * (U[1 + k] * inv));",
     "    for (int k = 0; k < 3; k++) dU[1 + k] = -(a * (U[1 + k] / U[0]));"),
    ("    dU[4] = -(a * (U[4] * inv));", "    dU[4] = -(a * (U[4] / U[0]));"),
    ("    for (int k = 0; k < 3; k++) acc[1 + k] = fma(-b, U[1 + k] * inv, acc[1 + k]);",
     "    for (int k = 0; k < 3; k++) acc[1 + k] = fma(-b, U[1 + k] / U[0], acc[1 + k]);"),
]


def _plain_source():
    src = open(SRC).read()
    for old, new in PLAIN:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    return src


@pytest.fixture(scope="module")
def plain_lib(tmp_path_factory):
    d = tmp_path_factory.mktemp("plain")
    c = os.path.join(d, "plain.c")
    lib = os.path.join(d, "libplain.so")
    open(c, "w").write(_plain_source())
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fexcess-precision=standard", "-fPIC", "-shared", "-o", lib, c, "-lm"])
    return lib


def _cases():
    out = []
    w = syn.make_workload("c1_32")
    out.append(("c1_32 supernovae", w["fb_params"], w["box"], w["state"], w["fb"], (1, 1, 1)))
    out.append(("c1_32 sinks", w["sink_params"], w["box"], w["state"], w["sink"], (1, 1, 1)))
    rng = np.random.default_rng(77)
    for n, g, rK, S, per in (((7, 7, 7), 3, 2.5, 3, (1, 1, 1)), ((9, 4, 5), 3, 3.0, 4, (0, 0, 0)),
                             ((8, 6, 7), 2, 1.5, 2, (1, 0, 1))):
        box = syn.Box(n, g)
        st = syn.gas_state(rng, box)
        parts = syn.particles(rng, n, 12, "feedback")
        out.append((f"edge {n} r_K {rK}", syn.feedback_params(r_K=rK, subsample=S), box, st, parts, per))
    box = syn.Box((20, 20, 20), 4)
    st = syn.gas_state(rng, box)
    out.append(("clustered 20^3 supernovae", syn.feedback_params(), box, st,
                syn.particles(rng, box.n, 400, "feedback", clustered=400, nclusters=2), (1, 1, 1)))
    st2 = syn.gas_state(rng, box)
    v = box.valid(st2)
    v[0] *= 3.0
    v[4] *= 3.0
    sk = syn.particles(rng, box.n, 60, "sink", clustered=60, nclusters=2)
    out.append(("clustered 20^3 sinks", syn.sink_params(dt=0.5), box, st2, sk, (1, 1, 1)))
    return out


def _run_cases(orc):
    res = []
    for name, params, box, state, parts, per in _cases():
        st = state.copy()
        pp = {k: v.copy() for k, v in parts.items()}
        r = orc.cycle(params, box, st, pp, periodic=per, want_abs=True, want_eta=True)
        res.append(dict(name=name, gathered=r["gathered"], buf=r["buf"], absbuf=r["absbuf"], eta=r["eta"],
                        state=st, parts=pp, state0=state))
    return res


def _vcom_scale(orc, params, box, state, parts, Msnr):
    """(sum_c omega_c |p_c| V + |p_ej|) / M_snr per axis and particle (V = 1)."""
    U = box.grid(state)
    g = box.g
    n = box.n
    out = np.zeros((3, len(parts["x"])))
    for s in range(len(parts["x"])):
        ijk, om = orc.kernel_of(params, box, parts["x"][s], parts["y"][s], parts["z"][s])
        for (i, j, k), w in zip(ijk, om):
            c = (k % n[2] + g, j % n[1] + g, i % n[0] + g)
            out[:, s] += w * np.abs(U[1:4, c[0], c[1], c[2]])
        out[:, s] = (out[:, s] + np.abs([parts["px"][s], parts["py"][s], parts["pz"][s]])) / Msnr[s]
    return out


def _omega_sum(orc, params, box, parts):
    """sum_s omega_s per valid cell (z, y, x)."""
    n = box.n
    out = np.zeros(n[::-1])
    for s in range(len(parts["x"])):
        ijk, om = orc.kernel_of(params, box, parts["x"][s], parts["y"][s], parts["z"][s])
        for (i, j, k), w in zip(ijk, om):
            out[k % n[2], j % n[1], i % n[0]] += w
    return out


def _flatten(res):
    out = {}
    for i, r in enumerate(res):
        for k in ("gathered", "buf", "absbuf", "eta", "state", "state0"):
            out[f"{i}_{k}"] = r[k]
        for k, v in r["parts"].items():
            out[f"{i}_p_{k}"] = v
    return out


_CHILD = (
    "import sys, numpy as np; sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r});"
    "import oracle; import test_oracle_plain_arith as t;"
    "res = t._run_cases(oracle); np.savez({out!r}, **t._flatten(res))"
)


def test_plain_source_differs_only_where_stated():
    src, plain = open(SRC).read(), _plain_source()
    assert src.count("fma(") >= 6 and plain.count("#define fma(a, b, c) ((a) * (b) + (c))") == 1
    assert "* inv" not in plain.replace("(0.5 * inv)", "")


@pytest.mark.slow
def test_every_pin_passes_with_separately_rounded_arithmetic(plain_lib):
    env = dict(os.environ, PMP_ORACLE_LIB=plain_lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider",
                        *PINS], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:]


def test_separately_rounded_oracle_agrees_to_rounding(orc, plain_lib, tmp_path):
    out = str(tmp_path / "plain.npz")
    env = dict(os.environ, PMP_ORACLE_LIB=plain_lib)
    code = _CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), out=out)
    subprocess.check_call([sys.executable, "-c", code], cwd=ROOT, env=env, timeout=600)
    other = np.load(out)
    mine = _run_cases(orc)
    report = {}
    for i, (case, r) in enumerate(zip(_cases(), mine)):
        name, params, box = case[0], case[1], case[2]
        g0, g1 = r["gathered"], other[f"{i}_gathered"]
        scale = np.abs(g0)
        if params["kind"] == "feedback":
            # v_COM = (sum omega p V + p_ej) / M_snr: its sum cancels, so its
            # rounding is measured against (sum omega |p| V + |p_ej|) / M_snr
            scale[2:5] = _vcom_scale(orc, params, box, r["state0"], case[4], g0[0])
        rel = np.abs(g0 - g1) / np.maximum(scale, 1e-300)
        assert np.all(rel <= 16 * EPS), (name, "gathered", float(rel.max()))
        nv = box.ncells_valid
        A = box.valid(r["absbuf"]).reshape(5, nv)
        D0 = box.valid(r["buf"]).reshape(5, nv)
        D1 = box.valid(other[f"{i}_buf"]).reshape(5, nv)
        dbuf = np.abs(D0 - D1)
        U0 = box.valid(r["state0"]).reshape(5, nv)
        dD = 8 * EPS * A
        if params["kind"] == "feedback":
            # Eq. du's momentum and energy rows carry v_COM, whose two
            # evaluations differ by dv (checked above): (rho + q) omega dv and
            # v_COM's share of the energy row, Pv omega |dv|, per contribution
            dv = np.abs(g0[2:5] - g1[2:5]).max(axis=1)
            Om = _omega_sum(orc, params, box, case[4]).reshape(nv)
            qmax, Pvmax = float(np.max(g0[8])), float(np.max(g0[10]))
            vmax = np.abs(g0[2:5]).max(axis=1)
            for a in range(3):
                # ... and the rounding of omega ((rho + q) v_COM - p) itself,
                # whose two terms cancel
                dD[1 + a] += Om * (U0[0] + qmax) * dv[a] + \
                    4 * EPS * Om * ((U0[0] + qmax) * vmax[a] + np.abs(U0[1 + a]))
            dD[4] += Om * Pvmax * float(np.sqrt(np.sum(dv * dv)))
        elif params["kind"] == "sink":
            # a = max(K w, rho - rho_Tr): where the Truelove term wins, rho_Tr's
            # rounding (its c_s^2 divides by rho) is eps rho_Tr ~ eps rho per
            # contribution, and every row carries a (times U_f / rho)
            Nc = _omega_sum(orc, params, box, case[4]).reshape(nv)
            for f in range(5):
                dD[f] += 8 * EPS * Nc * np.abs(U0[f])
        assert np.all(dbuf <= dD), (name, "buffer", np.argwhere(dbuf > dD)[:3].tolist(),
                                    float(np.max(dbuf / np.maximum(dD, 1e-300))))
        # sinks: the limiter's Truelove bound rho - rho_Tr differs by the
        # rounding of rho_Tr between the two evaluations
        dlim = 8 * EPS * np.abs(U0[0]) if params["kind"] == "sink" else None
        tol, amb = state_tolerance(params, U0, D0, A, r["eta"], tau=8 * EPS, dD=dD, dlim=dlim)
        ds = np.abs(box.valid(r["state"]).reshape(5, nv) - box.valid(other[f"{i}_state"]).reshape(5, nv))
        assert np.all(ds <= tol), (name, "state after Step 5", float(np.max(ds / np.maximum(tol, 1e-300))))
        if params["kind"] == "sink":
            from bounds import sink_return_tolerance

            p0 = case[4]
            vmax = float(np.max(np.abs(U0[1:4]) / U0[0]))
            R = int(np.ceil(params["r_K"]))
            tm, tp = sink_return_tolerance(p0["m"], r["parts"]["m"], r["parts"]["px"], vmax, (2 * R + 1) ** 3,
                                           tau=8 * EPS)
            for k in ("m", "px", "py", "pz"):
                d = np.abs(r["parts"][k] - other[f"{i}_p_{k}"])
                t = tm if k == "m" else sink_return_tolerance(p0["m"], r["parts"]["m"], r["parts"][k], vmax,
                                                              (2 * R + 1) ** 3, tau=8 * EPS)[1]
                assert np.all(d <= t), (name, k)
        report[name] = dict(buffer_values_differing=int(np.count_nonzero(dbuf)),
                            state_values_differing=int(np.count_nonzero(ds)))
    # the two evaluations are not the same function: rounding differs somewhere
    assert sum(v["buffer_values_differing"] for v in report.values()) > 0, json.dumps(report)
