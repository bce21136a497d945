"""The bench's host-side arithmetic, on the CPU: the roofline object of the
dominant kernel, the per-pass HBM figures and the clock record.  These are
pure functions of timings, sizes and sampled text, so they are checked here
with made-up inputs; the GPU only supplies the numbers."""
import os
import tempfile

import pytest

import bench
from paper_2509_18261_gb300 import synthetic as syn


def _box():
    return syn.Box((512, 512, 512), 4)


def test_alu_roofline_of_the_supernova_kernels():
    box = _box()
    pairs = {"fb": 491_934_207, "sink": 562_210_341}
    for kernel, per_pair in (("fb_deposit", 29), ("fb_plan_gather", 9)):  # Eq. du; the gather sums
        r = bench.roofline(kernel, 24.2, pairs, box, 14_680_064, 2_097_152, 6793.4, "measured")
        flops = per_pair * pairs["fb"]  # canonical FP64 operations per pair
        assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["peak"] == bench.FP64_PEAK_TFLOPS
        assert r["achieved"] == pytest.approx(flops / 24.2e-3 / 1e12, rel=1e-12)
        assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-12)
        assert r["kernel"] == kernel and r["ms_per_launch"] == 24.2


def test_alu_roofline_of_the_fused_sink_kernel():
    # Sec. 3.1.1 gather sums and weights (8) plus the accretion deposit (7) per pair
    box = _box()
    pairs = {"fb": 491_934_207, "sink": 562_210_341}
    r = bench.roofline("sink_gather_deposit", 23.3, pairs, box, 14_680_064, 2_097_152, 6793.4, "measured")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(15 * pairs["sink"] / 23.3e-3 / 1e12, rel=1e-12)


def test_algorithmic_bytes_of_the_supernova_kernels():
    n, pairs, ts, tb = 1000, 33_000, 20_000, 21_000
    assert bench.alg_bytes_fb("plan_gather", n, pairs, ts, tb) == 160 * n + 8 * pairs + 40 * ts
    assert bench.alg_bytes_fb("deposit", n, pairs, ts, tb) == 72 * n + 8 * pairs + 40 * ts + 80 * tb


def test_hbm_roofline_of_the_sink_apply():
    box = _box()
    r = bench.roofline("sink_apply", 7.2, {"fb": 1, "sink": 1}, box, 1, 1, 6793.4, "measured")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(128 * 512 ** 3 / 7.2e-3 / 1e9, rel=1e-12)
    assert r["frac"] == pytest.approx(r["achieved"] / 6793.4, rel=1e-12)


def test_hbm_roofline_of_the_zero_and_fold_passes():
    box = _box()
    ghosts = box.ncells_padded - 512 ** 3  # the 520^3 buffer less its valid cells
    r = bench.roofline("fb_fold", 0.27, {"fb": 1, "sink": 1}, box, 1, 1, 6793.4, "measured")
    assert r["bound"] == "hbm"
    assert r["achieved"] == pytest.approx(120 * ghosts / 0.27e-3 / 1e9, rel=1e-12)
    r = bench.roofline("sink_zero", 0.86, {"fb": 1, "sink": 1}, box, 1, 1, 6793.4, "measured")
    assert r["achieved"] == pytest.approx(40 * 520 ** 3 / 0.86e-3 / 1e9, rel=1e-12)
    out = bench.cell_pass_hbm({"sink_fold": (1.0, 0.27)}, box, 6793.4)
    assert out["sink_fold"]["bytes"] == 120 * ghosts


def test_traffic_is_reported_only_for_the_profiled_sources(monkeypatch):
    # the committed summary names the digest of the sources it was taken on
    import re

    txt = open(bench.os.path.join(bench.ROOT, "profiles", "counters_c5_192.md")).read()
    rows = [[c.strip() for c in line.strip().strip("|").split("|")] for line in txt.splitlines()]
    kernel = next(r[1] for r in rows if len(r) == 13 and r[1].startswith("fb_"))
    t = bench.profiled_traffic(kernel, 491934207)
    assert t is None or t > 1e10
    assert bench.profiled_traffic("no_such_kernel", 1000) is None
    # with the digest of the capture, the per-pair bytes scale with the pairs
    monkeypatch.setattr(bench, "src_digest", lambda: re.search(r"csrc_sha:\s*([0-9a-f]+)", txt).group(1))
    a = bench.profiled_traffic(kernel, 1000)
    assert a is not None and bench.profiled_traffic(kernel, 2000) == pytest.approx(2 * a)
    assert 20.0 < a / 1000 < 400.0  # bytes per pair of the 192^3 capture


def test_profiled_row_reads_the_binding_counters(monkeypatch):
    import re

    txt = open(bench.os.path.join(bench.ROOT, "profiles", "counters_c5_192.md")).read()
    monkeypatch.setattr(bench, "src_digest", lambda: re.search(r"csrc_sha:\s*([0-9a-f]+)", txt).group(1))
    rows = [[c.strip() for c in line.strip().strip("|").split("|")] for line in txt.splitlines()]
    names = [r[1] for r in rows if len(r) == 13 and r[1] != "bench name" and not r[1].startswith("---")]
    assert "fb_plan_gather" in names and "fb_deposit" in names
    for name in names:
        row = bench.profiled_row(name)
        assert row is not None
        for k in ("issue_pct", "fp64_pipe_pct", "dram_pct", "warps_active_pct"):
            assert 0.0 < row[k] <= 100.0
        assert row["fp64_per_unit"] >= 0.0 and row["bytes_per_unit"] > 0.0


def test_cell_pass_hbm_rates():
    box = _box()
    km = {"fb_apply": (1.0, 5.2), "sink_apply": (1.0, 7.2), "fb_zero": (1.0, 0.86), "sink_cell_records": (1.0, 4.4)}
    out = bench.cell_pass_hbm(km, box, 6793.4)
    assert out["fb_apply"]["ms"] == pytest.approx(5.2)
    assert out["fb_apply"]["GB/s"] == pytest.approx(120 * 512 ** 3 / 5.2e-3 / 1e9, rel=1e-3)
    assert out["fb_apply"]["frac"] == pytest.approx(out["fb_apply"]["GB/s"] / 6793.4, rel=1e-3)
    assert out["sink_apply"]["bytes"] == 128 * 512 ** 3
    assert out["sink_apply"]["ms"] == pytest.approx(7.2)
    assert out["fb_zero"]["bytes"] == 40 * box.ncells_padded
    # state read (40 B), then the 32-byte G and D records and three dense 8-byte arrays written
    assert out["sink_cell_records"]["bytes"] == (40 + 32 + 32 + 3 * 8) * 512 ** 3
    assert "sink_spread" not in out  # a pass that was not timed is left out


def test_source_digest_follows_code_not_comments(tmp_path):
    src = 'int a; // sum\n/* two\n   lines */ const char *s = "//x";\n\nchar q = \'"\';  \n'
    (tmp_path / "k.cu").write_text(src)
    base = bench.src_digest(str(tmp_path))
    (tmp_path / "k.cu").write_text(src.replace("// sum", "// total").replace("two", "three") + "\n// more\n")
    assert bench.src_digest(str(tmp_path)) == base
    (tmp_path / "k.cu").write_text(src.replace('"//x"', '"//y"'))  # inside a string literal: code
    assert bench.src_digest(str(tmp_path)) != base
    (tmp_path / "k.cu").write_text(src.replace("int a;", "int b;"))
    assert bench.src_digest(str(tmp_path)) != base
    (tmp_path / "k.cu").write_text(src)
    (tmp_path / "pmp_batch.cu").write_text("int z;")  # excluded: not a single-box kernel source
    assert bench.src_digest(str(tmp_path)) == base
    assert bench.code_of(src) == 'int a;\n  const char *s = "//x";\nchar q = \'"\';'


def test_batched_hbm_view_counts_zero_fold_and_apply_per_pass():
    # one 16^3 patch with 4 ghost cells per side: 24^3 buffer cells
    v, p = 16 ** 3, 24 ** 3
    out = bench.batched_hbm_view(v, p, 2.0, 6800.0, "measured")
    per_pass = 40 * p + 120 * (p - v) + 120 * v
    assert out["algorithmic_bytes_per_cycle"] == 2 * per_pass
    assert out["GB/s"] == pytest.approx(2 * per_pass / 2e-3 / 1e9)
    assert out["frac"] == pytest.approx(out["GB/s"] / 6800.0)
    assert out["peak_source"] == "measured"


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _clocks_from(lines):
    c = bench.Clocks(0)
    fd, c.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(lines) + "\n")
    c.proc = _Done()
    return c.stop()


def test_clock_record_median_and_reasons():
    rows = [
        "0, 2070, 2070, 1100.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    ]
    r = _clocks_from(rows)
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]


def test_clock_record_flags_thermal_slowdown_and_skips_bad_rows():
    rows = [
        "0, 1500, 2070, 1400.0, 0x0000000000000040, Not Active, Active, Not Active, Not Active",
        "0, [N/A], 2070, 1400.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
    ]
    r = _clocks_from(rows)
    assert r["sm_mhz"] == 1500.0 and r["samples"] == 2
    assert r["reasons"] == ["hw_thermal_slowdown"]


def test_cpu_baseline_leg_runs_the_oracle(orc):
    import argparse

    r = bench.cpu_baseline(argparse.Namespace(cpu_sample_n=16))
    assert r["kind"] == "oracle" and r["cores"] == 1 and r["host_cpus"] >= 1
    assert r["value"] > 0 and r["unit"] == "particles/s" and "16^3" in r["sample"]
