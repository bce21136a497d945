"""The seeded input generators (paper_2509_18261_gb300/synthetic.py) draw what
the stated recipe says, checked against closed forms of the distributions:
lognormal gas with Gaussian momenta at uniform specific thermal energy,
Plummer clusters (cumulative mass r^3 / (r^2 + a^2)^(3/2)), power-law patch
counts (density of X proportional to X^-2), log-uniform masses, the mixed
workload's split, positions inside [0, n) and the same arrays for the same
seed.  Sample sizes make each tolerance several standard errors wide."""
import math

import numpy as np

from paper_2509_18261_gb300 import synthetic as syn


def test_gas_recipe():
    box = syn.Box((48, 48, 48), 2)
    st = syn.gas_state(np.random.default_rng(1), box)
    v = box.valid(st).reshape(5, -1)
    lr = np.log(v[0])
    assert abs(lr.mean() + 0.5) < 0.02 and abs(lr.std() - 1.0) < 0.02  # ln rho ~ N(-1/2, 1)
    assert abs(v[0].mean() - 1.0) < 0.03  # mean density 1
    for f in (1, 2, 3):
        assert abs(v[f].mean()) < 0.002 and abs(v[f].std() - 0.1) < 0.002
    eint = v[4] - (v[1] ** 2 + v[2] ** 2 + v[3] ** 2) / (2.0 * v[0])
    assert np.allclose(eint, v[0], rtol=1e-12, atol=0)  # specific thermal energy 1
    assert np.all(np.isnan(box.grid(st)[:, 0]))  # ghost cells are never meant to be read


def test_plummer_clusters_follow_the_plummer_mass_profile():
    n, a, count = (4096, 4096, 4096), 2.0, 200_000  # a box large enough that nothing wraps
    pos = syn._plummer_positions(np.random.default_rng(7), 1, count, a, n)
    centre = syn._uniform_positions(np.random.default_rng(7), 1, n)[:, 0]  # drawn first
    d = pos - centre[:, None]
    r = np.sqrt((d * d).sum(axis=0))
    for x in (0.5, 1.0, 2.0, 4.0):
        want = x ** 3 / (x * x + 1.0) ** 1.5  # M(< x a) / M
        assert abs(np.mean(r < x * a) - want) < 0.005, x
    assert np.all(np.abs((d / r).mean(axis=1)) < 0.01)  # isotropic directions


def test_power_law_patch_counts():
    xmax = 20001.0
    cnt = syn.power_law_counts(np.random.default_rng(3), 400_000, xmax)
    assert cnt.min() >= 0 and cnt.max() <= xmax - 2
    for k in (1, 3, 9, 99):
        x = k + 1.0  # n >= k  <=>  X >= k + 1
        want = (1.0 / x - 1.0 / xmax) / (1.0 - 1.0 / xmax)
        assert abs(np.mean(cnt >= k) - want) < 4 * math.sqrt(want * (1 - want) / cnt.size) + 1e-4, k


def test_particle_masses_and_positions():
    n = (64, 48, 32)
    fb = syn.particles(np.random.default_rng(4), n, 100_000, "feedback", clustered=50_000, nclusters=10)
    sk = syn.particles(np.random.default_rng(5), n, 100_000, "sink")
    for p, lo, hi in ((fb, 1e-3, 1e-1), (sk, 1.0, 100.0)):
        lm = np.log(p["m"])
        assert lm.min() >= math.log(lo) and lm.max() <= math.log(hi)
        assert abs(lm.mean() - 0.5 * (math.log(lo) + math.log(hi))) < 0.02  # log-uniform
        for a, key in enumerate(("x", "y", "z")):
            assert p[key].min() >= 0.0 and p[key].max() < n[a]
        v = p["px"] / p["m"]
        assert abs(v.std() - 0.1) < 0.002
    assert np.all(fb["e"] == 1.0)


def test_mixed_workload_split_and_determinism():
    w = syn.make_workload("c5_512", n=32, count_scale=(32 / 512) ** 3)
    spec = syn.WORKLOADS["c5_512"]["mixed"]
    assert spec["count"] == 512 ** 3 // 8 and spec["clustered"] * 4 == spec["count"]
    total = len(w["fb"]["x"]) + len(w["sink"]["x"])
    assert total == 4096 and len(w["sink"]["x"]) * 8 == total  # 7/8 supernovae, 1/8 sinks
    w2 = syn.make_workload("c5_512", n=32, count_scale=(32 / 512) ** 3)
    for kind in ("fb", "sink"):
        for k, v in w[kind].items():
            assert np.array_equal(v, w2[kind][k])
    assert np.array_equal(w["state"], w2["state"], equal_nan=True)
