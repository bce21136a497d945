"""The ROUNDED deposit (App. A.1 reproducible atomics) on the GPU, through the
C ABI, against the oracle's index-order deposit.

- values reached by one particle: the GPU's rounded buffer equals the
  oracle's bit for bit (E = eps |v| in any order);
- every other value is the GPU's sum with low significand bits cleared: it
  lies within the dropped quantum plus the atomic-order tolerance of the
  oracle's plain sum;
- two particle orders on the GPU agree on every single-contributor value;
- pmp_set_rounding_margin rejects margins outside [0, 104].
"""
import numpy as np
import pytest

from paper_2509_18261_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


def _case(seed, n=16, count=1200, clustered=600, ncl=6):
    rng = np.random.default_rng(seed)
    box = syn.Box((n, n, n), 4)
    state = syn.gas_state(rng, box)
    parts = syn.particles(rng, box.n, count, "feedback", clustered=clustered, nclusters=ncl)
    return rng, box, state, parts


def _gpu_rounded(params, box, state, parts, M):
    import torch

    from paper_2509_18261_gb300 import pmp

    st = torch.from_numpy(state.copy()).cuda()
    pd = pmp.parts_to_device(parts)
    ps = pmp.Pass(params, box, st, pd, mode="rounded")
    pmp.pmp_set_rounding_margin(ps.ctx, M)
    ps.run(stop_after="deposit")
    torch.cuda.synchronize()
    buf = ps.buffer.data.cpu().numpy()
    err = pmp.pmp_get_error(ps.ctx)
    ps.ctx.close()
    assert err == (0, -1)
    return buf


def _oracle(orc, params, box, state, parts, M):
    G = orc.gather(params, box, state, parts)
    plain, absb = box.empty(0.0), box.empty(0.0)
    orc.deposit(params, box, state, parts, G, plain, absb)
    rounded = box.empty(0.0)
    E = orc.deposit_rounded(params, box, state, parts, G, rounded, M)
    return plain, absb, rounded, E


def _contributions(orc, params, box, state, parts):
    """Number of particles adding to each buffer value (every field of a
    kernel cell), from the oracle's per-particle kernel lists."""
    cnt = box.empty(0.0)
    view = box.grid(cnt)
    g = box.g
    for s in range(len(parts["x"])):
        one = {k: v[s:s + 1] for k, v in parts.items()}
        ijk, _ = orc.deltas(params, box, state, one)
        for i, j, k in ijk:
            view[:, k + g, j + g, i + g] += 1.0
    return cnt


def _quantum(v, e, M):
    """Upper bound of the dropped amount: 2^N_bit units in the last place of
    v, N_bit of App. A.1 taken from e (clamped to [0, 52])."""
    out = np.zeros_like(v)
    ok = (v != 0) & (e > 0)
    r = e[ok] / np.abs(v[ok])
    m, k = np.frexp(r)
    nb = np.clip(np.where(m == 0.5, k - 1, k) + 52 + M, 0, 52)
    _, ev = np.frexp(np.abs(v[ok]))
    out[ok] = np.ldexp(1.0, ev - 53 + nb)
    return out


@pytest.mark.parametrize("M", [8, 28])
def test_rounded_deposit_against_oracle(orc, M):
    _, box, state, parts = _case(seed=11)
    params = syn.feedback_params()
    got = _gpu_rounded(params, box, state, parts, M)
    plain, absb, rounded, E = _oracle(orc, params, box, state, parts, M)
    single = (E > 0) & (E == EPS * np.abs(plain))
    multi = (E > 0) & ~single
    assert single.sum() > 1000 and multi.sum() > 1000
    assert np.array_equal(got.view(np.uint64)[single], rounded.view(np.uint64)[single])
    assert np.all(got[E == 0] == 0.0)
    # in any order every partial sum is at most sum |dU|, so the GPU's E is at
    # most (additions) eps sum |dU|: that bounds its dropped quantum; then
    # allow the atomic-order difference of the plain sum
    n = _contributions(orc, params, box, state, parts)
    tol = _quantum(plain, n * EPS * absb, M) + 1e-12 * absb
    assert np.all(np.abs(got - plain)[multi] <= tol[multi])
    assert np.all(np.abs(got) <= np.abs(plain) + 1e-12 * absb)


def test_two_orders_on_the_gpu(orc):
    rng, box, state, parts = _case(seed=13)
    params = syn.feedback_params()
    perm = rng.permutation(len(parts["x"]))
    p2 = {k: v[perm].copy() for k, v in parts.items()}
    a = _gpu_rounded(params, box, state, parts, 28)
    b = _gpu_rounded(params, box, state, p2, 28)
    _, _, _, E = _oracle(orc, params, box, state, parts, 28)
    plain = box.empty(0.0)
    orc.deposit(params, box, state, parts, orc.gather(params, box, state, parts), plain)
    single = (E > 0) & (E == EPS * np.abs(plain))
    assert np.array_equal(a.view(np.uint64)[single], b.view(np.uint64)[single])
    multi = (E > 0) & ~single
    differ = np.count_nonzero((a.view(np.uint64) != b.view(np.uint64)) & multi)
    assert differ < 0.5 * multi.sum()


def test_rounding_margin_is_checked():
    from paper_2509_18261_gb300 import pmp

    ctx = pmp.Context(syn.feedback_params())
    for bad in (-1, 105):
        with pytest.raises(pmp.PMPError):
            pmp.pmp_set_rounding_margin(ctx, bad)
    pmp.pmp_set_rounding_margin(ctx, 0)
    pmp.pmp_set_rounding_margin(ctx, 104)
    ctx.close()


def test_rounded_sink_deposit_against_oracle(orc):
    """Sinks in the ROUNDED mode: single-contributor values bit for bit, the
    rest within the dropped quantum of the oracle's plain sum."""
    import torch

    from paper_2509_18261_gb300 import pmp

    rng = np.random.default_rng(21)
    box = syn.Box((12, 12, 12), 4)
    state = syn.gas_state(rng, box)
    parts = syn.particles(rng, box.n, 24, "sink", clustered=12, nclusters=2)
    params = syn.sink_params(dt=0.05)
    st = torch.from_numpy(state.copy()).cuda()
    pd = pmp.parts_to_device(parts)
    ps = pmp.Pass(params, box, st, pd, mode="rounded")
    ps.run(stop_after="deposit")
    torch.cuda.synchronize()
    got = ps.buffer.data.cpu().numpy()
    assert pmp.pmp_get_error(ps.ctx) == (0, -1)
    ps.ctx.close()
    plain, absb, rounded, E = _oracle(orc, params, box, state, parts, 28)
    # one pair per value: its E is eps |value| in any order.  (E == eps |sum|
    # does not single these out here: a sink pair whose removal is exactly 0,
    # w underflowing where rho < rho_Tr, adds nothing to the first E but
    # doubles it when it comes second.)
    n = _contributions(orc, params, box, state, parts)
    single = (E > 0) & (n == 1)
    multi = (E > 0) & (n > 1)
    assert single.sum() > 100 and multi.sum() > 100
    assert np.array_equal(got.view(np.uint64)[single], rounded.view(np.uint64)[single])
    tol = _quantum(plain, n * EPS * absb, 28) + 1e-12 * absb
    assert np.all(np.abs(got - plain)[multi] <= tol[multi])
