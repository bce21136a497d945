"""Pins of the oracle's auxiliary fields under accretion (Sec. 3.1.1: the
dual-energy internal energy and passive scalars keep their value per unit
mass, Delta rho_sp = (rho_sp / rho) Delta rho):

- concentration invariance: X_new / rho_new = X_old / rho_old to rounding in
  every cell the pass changes, and cells it does not change keep X bit for
  bit;
- a species with concentration 1 (X = rho) stays equal to the density
  bit for bit;
- a species with concentration 0 stays 0.
"""
import numpy as np

from paper_2509_18261_gb300 import synthetic as syn


def _sink_pass_with_extra(orc, box, state, parts, params, X):
    G = orc.gather(params, box, state, parts)
    buf = box.empty(0.0)
    orc.deposit(params, box, state, parts, G, buf)
    orc.fold(box, buf)
    orc.apply_extra(params, box, state, buf, X)
    orc.return_sinks(params, box, state, buf, parts, G)
    orc.apply(params, box, state, buf)
    return buf


def test_concentrations_are_kept(orc):
    rng = np.random.default_rng(12)
    box = syn.Box((14, 12, 10), 4)
    state = syn.gas_state(rng, box)
    box.valid(state)[:] *= 3.0  # denser gas: the limiter engages in some cells
    parts = syn.particles(rng, box.n, 12, "sink")
    params = syn.sink_params(dt=1.0)
    X = np.zeros((4, box.field_stride))
    rho0 = state[0].copy()
    X[0] = rho0 * rng.uniform(0.0, 1.0, box.field_stride)  # a species
    X[1] = rho0 * 1.5                                       # internal energy density, e_int,sp = 1.5
    X[2] = rho0                                             # concentration 1
    X[3] = 0.0                                              # concentration 0
    X0 = X.copy()
    st = state.copy()
    buf = _sink_pass_with_extra(orc, box, st, {k: v.copy() for k, v in parts.items()}, params, X)
    v = lambda a: box.valid(a.reshape(1, -1))[0]  # noqa: E731
    touched = np.any(box.valid(buf) != 0, axis=0)
    assert touched.sum() > 500
    rho_new, rho_old = box.valid(st)[0], box.valid(state)[0]
    assert np.any(rho_new[touched] != rho_old[touched])
    for f in (0, 1):
        c_old = v(X0[f]) / rho_old
        c_new = v(X[f]) / rho_new
        assert np.allclose(c_new[touched], c_old[touched], rtol=8 * 2.0 ** -52, atol=0)
        assert np.array_equal(v(X[f])[~touched], v(X0[f])[~touched])
    assert np.array_equal(v(X[2]), rho_new)
    assert np.all(X[3] == 0.0)
