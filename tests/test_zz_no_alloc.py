"""pmp_deposit_noalloc, the Step-1 entry point for callers that cannot
allocate device memory (code inside another framework's memory pool, plugins
handed only pre-allocated buffers), against the regular entry points
pmp_gather + pmp_deposit, through the C ABI, on two calls in a row.

The allocation-free call keeps its plan in a fixed scratch array inside the
library, so two calls in a row also check that the second call does not see
stale contents from the first.
"""
import numpy as np
import pytest

from paper_2509_18261_gb300 import synthetic as syn
from helpers import assert_bits_equal, assert_within_abs

pytestmark = pytest.mark.gpu


def _inputs():
    w = syn.make_workload("c1_32")
    rng = np.random.default_rng(20261203)
    parts = syn.particles(rng, w["box"].n, 6000, "feedback", clustered=2400, nclusters=6)
    return w["box"], w["state"], parts, syn.feedback_params()


def test_noalloc_matches_regular_entry_points_on_two_calls(orc):
    import torch

    from paper_2509_18261_gb300 import pmp

    box, state, parts, params = _inputs()
    n = len(parts["x"])
    # oracle sums of |dU| per cell: the tolerance of atomic accumulation
    G_ref = orc.gather(params, box, state, parts)
    buf_ref, abs_ref = box.empty(0.0), box.empty(0.0)
    orc.deposit(params, box, state, parts, G_ref, buf_ref, abs_ref)
    A = box.grid(abs_ref)

    st = torch.from_numpy(state).cuda()
    pd = pmp.parts_to_device(parts)
    ps = pmp.Pass(params, box, st, pd, mode="atomic")
    ps.run(stop_after="deposit")
    torch.cuda.synchronize()
    reg_g = ps.gathered_view().cpu().numpy()
    reg_buf = box.grid(ps.buffer.data.cpu().numpy())
    assert_within_abs(reg_buf, box.grid(buf_ref), A, "regular entry points vs oracle")

    for call in range(2):
        buf = pmp.Mesh(torch.zeros((5, box.field_stride), dtype=torch.float64, device="cuda"), box.n, box.g)
        g = torch.full((12, n), float("nan"), dtype=torch.float64, device="cuda")
        pmp.pmp_deposit_noalloc(params, ps.state, pd, g, buf)
        torch.cuda.synchronize()
        assert_bits_equal(g.cpu().numpy(), reg_g, f"gathered rows, call {call + 1}")
        got = box.grid(buf.data.cpu().numpy())
        assert_within_abs(got, reg_buf, 2.0 * A, f"buffer vs regular entry points, call {call + 1}")
        assert_within_abs(got, box.grid(buf_ref), A, f"buffer vs oracle, call {call + 1}")
    ps.ctx.close()


def test_noalloc_rejects_more_particles_than_its_scratch_holds():
    import torch

    from paper_2509_18261_gb300 import pmp

    box, state, _, params = _inputs()
    n = 200_000  # 200k x (28 + 8 * 81) bytes > 64 MiB at r_K = 2
    z = torch.zeros(n, dtype=torch.float64, device="cuda") + 1.0
    big = {k: z for k in ("x", "y", "z", "m", "px", "py", "pz", "e")}
    st = pmp.Mesh(torch.from_numpy(state).cuda(), box.n, box.g)
    buf = pmp.Mesh(torch.zeros((5, box.field_stride), dtype=torch.float64, device="cuda"), box.n, box.g)
    g = torch.zeros((12, n), dtype=torch.float64, device="cuda")
    with pytest.raises(pmp.PMPError) as e:
        pmp.pmp_deposit_noalloc(params, st, big, g, buf)
    assert e.value.code == 6
    assert torch.count_nonzero(buf.data).item() == 0


def test_noalloc_skips_particles_outside_the_box(orc):
    """Particles outside [0, n) (or with a NaN position) receive zero gathered
    rows and deposit nothing; the others deposit as if alone."""
    import torch

    from paper_2509_18261_gb300 import pmp

    box, state, parts, params = _inputs()
    inside = {k: v[:500].copy() for k, v in parts.items()}
    mixed = {k: v[:520].copy() for k, v in parts.items()}
    n = box.n
    bad = [(n[0] + 0.5, 1.0, 1.0), (-0.25, 3.0, 3.0), (1.0, float(n[1]), 1.0), (2.0, 2.0, -1e-300),
           (float("nan"), 1.0, 1.0)]
    for r in range(20):
        x, y, z = bad[r % len(bad)]
        mixed["x"][500 + r], mixed["y"][500 + r], mixed["z"][500 + r] = x, y, z
    G_ref = orc.gather(params, box, state, inside)
    buf_ref, abs_ref = box.empty(0.0), box.empty(0.0)
    orc.deposit(params, box, state, inside, G_ref, buf_ref, abs_ref)
    st = pmp.Mesh(torch.from_numpy(state).cuda(), box.n, box.g)
    pd = pmp.parts_to_device(mixed)
    for call in range(2):
        buf = pmp.Mesh(torch.zeros((5, box.field_stride), dtype=torch.float64, device="cuda"), box.n, box.g)
        g = torch.full((12, 520), float("nan"), dtype=torch.float64, device="cuda")
        pmp.pmp_deposit_noalloc(params, st, pd, g, buf)
        torch.cuda.synchronize()
        gn = g.cpu().numpy()
        assert_bits_equal(gn[:, :500], G_ref, f"gathered rows of the particles inside, call {call + 1}")
        assert np.all(gn[:, 500:] == 0.0), "particles outside get zero rows"
        assert_within_abs(box.grid(buf.data.cpu().numpy()), box.grid(buf_ref), box.grid(abs_ref),
                          f"buffer: only the particles inside deposit, call {call + 1}")
