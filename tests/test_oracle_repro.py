"""Pins of the oracle's reproducible-atomics deposit (App. A.1 of He et al.
2025) to facts that do not come from the oracle itself.

- A value reached by one particle has E = eps |v| exactly, so the printed
  rule keeps all but the M least significant bits of the plain sum.
- Rounding only clears low significand bits (truncation toward zero).
- E bounds the change of a buffer value under re-ordering (App. A.1, step
  2: "an upper limit on the amount by which the sum could be changed").
- With the two orders' dropped-bit counts equal, two orders disagree only
  where the sum lies within the re-ordering change of a rounding boundary,
  about 2^-M of the values (App. A.1); E itself depends on the order, and
  the share of values whose dropped-bit count differs is measured, not
  assumed.
"""
import numpy as np
import pytest

from paper_2509_18261_gb300 import synthetic as syn

EPS = 2.0 ** -52


def _case(seed=3, n=16, count=1200, clustered=600, ncl=6):
    rng = np.random.default_rng(seed)
    box = syn.Box((n, n, n), 4)
    state = syn.gas_state(rng, box)
    parts = syn.particles(rng, box.n, count, "feedback", clustered=clustered, nclusters=ncl)
    return rng, box, state, parts


def _deposit(orc, params, box, state, parts, M):
    G = orc.gather(params, box, state, parts)
    plain = box.empty(0.0)
    orc.deposit(params, box, state, parts, G, plain)
    rounded = box.empty(0.0)
    E = orc.deposit_rounded(params, box, state, parts, G, rounded, M)
    return plain, rounded, E


def test_single_contributor_keeps_all_but_M_bits(orc):
    box = syn.Box((12, 12, 12), 4)
    rng = np.random.default_rng(1)
    state = syn.gas_state(rng, box)
    parts = syn.particles(rng, box.n, 1, "feedback")
    for M in (0, 5, 28, 52):
        plain, rounded, E = _deposit(orc, syn.feedback_params(), box, state, parts, M)
        touched = E > 0
        assert touched.sum() > 50
        assert np.array_equal(E[touched], EPS * np.abs(plain[touched]))
        mask = np.uint64((1 << M) - 1)
        want = plain.view(np.uint64) & ~mask
        assert np.array_equal(rounded.view(np.uint64)[touched], want[touched])
        assert np.all(rounded[~touched] == 0.0)


def test_rounding_clears_low_bits_only(orc):
    _, box, state, parts = _case()
    plain, rounded, E = _deposit(orc, syn.feedback_params(), box, state, parts, 12)
    u, r = plain.view(np.uint64), rounded.view(np.uint64)
    assert np.all((r & ~u) == 0)  # no bit set that the plain sum does not have
    x = u ^ r  # bits the rounding cleared; all of them below some bit k ...
    m = x.copy()
    for sh in (1, 2, 4, 8, 16, 32):
        m |= m >> np.uint64(sh)  # m = 2^k - 1 with k the bit length of x
    assert np.all((r & m) == 0)  # ... and r keeps no bit below k
    assert np.all(x < np.uint64(1 << 52))
    assert np.all(np.abs(rounded) <= np.abs(plain))
    assert np.all(np.signbit(rounded) == np.signbit(plain))


def test_E_bounds_the_change_under_reordering(orc):
    rng, box, state, parts = _case(seed=5)
    params = syn.feedback_params()
    perm = rng.permutation(len(parts["x"]))
    p2 = {k: v[perm].copy() for k, v in parts.items()}
    a, _, E1 = _deposit(orc, params, box, state, parts, 28)
    b, _, E2 = _deposit(orc, params, box, state, p2, 28)
    assert np.count_nonzero(a != b) > 100  # the orders really differ
    assert np.all(np.abs(a - b) <= E1 + E2)


def _nbit(v, e, M):
    """Dropped-bit count of App. A.1 for each value (the same reading as the
    oracle's: ceil(log2(e/|v|)) + 52 + M, clamped to [0, 52])."""
    out = np.zeros(v.shape, dtype=np.int64)
    ok = (v != 0) & (e > 0)
    r = e[ok] / np.abs(v[ok])
    m, k = np.frexp(r)
    c = np.where(m == 0.5, k - 1, k)
    out[ok] = np.clip(c + 52 + M, 0, 52)
    return out


@pytest.mark.parametrize("M", [4, 8])
def test_orders_agree_up_to_boundary_cases(orc, M):
    rng, box, state, parts = _case(seed=7, n=20, count=3000, clustered=1500, ncl=6)
    params = syn.feedback_params()
    perm = rng.permutation(len(parts["x"]))
    p2 = {k: v[perm].copy() for k, v in parts.items()}
    a, ra, Ea = _deposit(orc, params, box, state, parts, M)
    b, rb, Eb = _deposit(orc, params, box, state, p2, M)
    multi = (Ea > 1.5 * EPS * np.abs(a)) & (a != 0)
    same_n = _nbit(a, Ea, M) == _nbit(b, Eb, M)
    differ = ra.view(np.uint64) != rb.view(np.uint64)
    sel = multi & same_n
    assert sel.sum() > 5000
    rate = np.count_nonzero(differ & sel) / sel.sum()
    # a value changes rounding interval only if it lies within |a - b| of a
    # boundary: at most about 2^-M of the values, well below at large M
    assert rate <= 2.0 * 2.0 ** -M
    # E depends on the order (App. A.1 sums eps times partial sums), so the
    # dropped-bit count itself differs for a measurable share of the values
    share = np.count_nonzero(multi & ~same_n) / multi.sum()
    assert 0.0 < share < 0.5
