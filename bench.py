"""Benchmark of the particle-mesh-particle (PMP) cycle on GB300.

One step = one full mixed cycle on the 512^3 workload: the supernova pass
(gather, deposit, fold, limited apply; Sec. 3.2.1) then the sink pass on the
updated state (gather, deposit, fold, Step-4 return, limited apply;
Sec. 3.1.1), atomic accumulation.  Every step starts from the same gas state
and sink masses/momenta (a device copy of the initial ones, 5.7 GB, counted
in the step's time), so every timed step does the same work.  Inputs
(state + buffer 11.2 GB) are larger than L2.

    python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]

Prints one JSON line.  With N > 1 (torchrun, one rank per GPU) every rank
runs an independent replica of the workload (weak scaling; the cycle has no
exchange step on one GPU) and the slowest rank's time is reported.
``--impl reference`` times the CPU oracle (the reference arm of this build)
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PMP cycle particles/s & cells/s on 1 GB300, % HBM roofline, fwd+bwd time"
WORKLOAD = "c5_512"
FP64_PEAK_TFLOPS = 1.25  # nominal dense FP64 of GB300 (fused multiply-add counted as 2)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--mode", default="atomic", choices=["atomic", "sorted"])
    ap.add_argument("--e2e-steps", type=int, default=None, help="end-to-end steps (default: --steps)")
    ap.add_argument("--copy-streams", type=int, default=4,
                    help="copy streams per direction in the pipelined end-to-end leg")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--cpu-sample-n", type=int, default=128)
    ap.add_argument("--n", type=int, default=None,
                    help="shrink the box to n^3 at equal particle density (profiling captures)")
    ap.add_argument("--keep-cluster-size", action="store_true",
                    help="with --n: fewer clusters of the full size instead of as many smaller ones")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------

def dist_init():
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, value):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        finally:
            os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# algorithmic work of one cycle (for the roofline)
# ---------------------------------------------------------------------------

def kernel_cell_count(parts, n, rK, chunk=1 << 20):
    """Number of (particle, kernel cell) pairs: cell centres strictly inside r_K
    (the per-pair unit of the particle kernels)."""
    import torch

    R = int(math.ceil(rK))
    o = torch.arange(-R, R + 1, device="cuda", dtype=torch.float64)
    total = 0
    N = parts["x"].numel()
    for s0 in range(0, N, chunk):
        d2 = None
        for a, key in enumerate(("x", "y", "z")):
            x = parts[key][s0:s0 + chunk]
            d = (torch.floor(x)[:, None] + o[None, :] + 0.5) - x[:, None]
            sq = d * d
            shape = [x.numel(), 1, 1, 1]
            shape[3 - a] = 2 * R + 1
            sq = sq.reshape(shape)
            d2 = sq if d2 is None else d2 + sq
        total += int((d2 < rK * rK).sum().item())
    return total




# Algorithmic work per kernel launch.  Particle kernels: canonical FP64
# operations per (particle, kernel cell) pair; cell kernels: bytes a perfect
# implementation moves.  See the kernel table of the design notes.
FLOPS_PER_PAIR = {"fb_gather": 9, "fb_plan_gather": 9, "fb_deposit": 29, "sink_gather": 8,
                  "sink_deposit": 7, "sink_gather_deposit": 15, "sink_return": 14}
FP32_PEAK_TOPS = 36.9  # measured FP32 instruction rate of this GB300 (dependent-free FFMA stream)


def roofline(kernel, ms, pairs, box, n_fb, n_sk, hbm_peak, peak_src):
    kind, stage = kernel.split("_", 1)
    nvalid = box.ncells_valid
    hbm_bytes = {
        "zero": 40 * box.ncells_padded,
        "fold": 120 * (box.ncells_padded - nvalid),
        "apply": 120 * nvalid + (8 * nvalid if kind == "sink" else 0),
        "cell_records": (40 + 88) * nvalid,
    }
    if stage == "plan":
        # FP32 decisions: 2 adds per candidate cell and per omega sub-point
        W = 2 * (2 if kind == "fb" else 4) + 1
        S3 = 64 if kind == "fb" else 0
        nparts = n_fb if kind == "fb" else n_sk
        ops = 2 * W ** 3 * nparts + 2 * S3 * pairs[kind]
        achieved = ops / (ms * 1e-3) / 1e12
        r = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TOPS, "unit": "Tops/s (FP32)",
             "frac": achieved / FP32_PEAK_TOPS, "peak_source": "measured FP32 issue rate"}
    elif stage in hbm_bytes:
        achieved = hbm_bytes[stage] / (ms * 1e-3) / 1e9
        r = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
             "peak_source": peak_src}
    else:
        flops = FLOPS_PER_PAIR.get(kernel, 0) * pairs[kind]
        achieved = flops / (ms * 1e-3) / 1e12
        r = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
             "frac": achieved / FP64_PEAK_TFLOPS, "peak_source": "nominal FP64, 152 SMs x 2 DFMA/clk x 2.07 GHz"}
    r["kernel"] = kernel
    r["ms_per_launch"] = ms
    units = pairs.get(kind) if stage not in hbm_bytes and stage != "plan" else nvalid
    r["traffic"] = profiled_traffic(kernel, units)
    return r


def cell_pass_hbm(kernel_ms, box, hbm_peak):
    """Per-launch HBM rate of the cell passes: algorithmic bytes (what a
    perfect implementation moves) over the CUDA-event time of the launch, and
    the fraction of the measured copy bandwidth.  The supernova apply reads
    the state and the summed change and writes the state (120 B per valid
    cell); the sink apply computes eta and updates the state in one pass (128
    B per valid cell with the eta it records for Step 4)."""
    nvalid, npad = box.ncells_valid, box.ncells_padded
    phases = {
        "fb_zero": (("fb_zero",), 40 * npad),
        "fb_fold": (("fb_fold",), 120 * (npad - nvalid)),
        "fb_apply": (("fb_apply",), 120 * nvalid),
        "sink_zero": (("sink_zero",), 40 * npad),
        "sink_cell_records": (("sink_cell_records",), (40 + 88) * nvalid),
        "sink_spread": (("sink_spread",), 136 * npad),
        "sink_fold": (("sink_fold",), 120 * (npad - nvalid)),
        "sink_apply": (("sink_apply",), 128 * nvalid),
    }
    out = {}
    for name, (kernels, nbytes) in phases.items():
        if not all(k in kernel_ms for k in kernels):
            continue
        ms = sum(kernel_ms[k][1] for k in kernels)
        gbs = nbytes / (ms * 1e-3) / 1e9
        out[name] = {"ms": round(ms, 4), "bytes": nbytes, "GB/s": round(gbs, 1), "frac": round(gbs / hbm_peak, 4)}
    return out


# Sources that neither define nor launch the single-box kernels the traffic
# figures are taken from: the batched form and its exchange plan, the
# allocation-free entry point and the peak probes.
DIGEST_EXCLUDES = ("pmp_batch.cu", "pmp_noalloc.cu", "pmp_probe.cu", "pmp_exchange.cu")


def code_of(text):
    """C/C++/CUDA source without its comments, trailing blanks and empty
    lines: what a compiler sees of it, up to layout.  String and character
    literals are kept as they are (a // or /* inside one is not a comment)."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            out.append(" ")
            i = n if j < 0 else j + 2
        elif c in "\"'":
            j = i + 1
            while j < n and text[j] != c and text[j] != "\n":
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    lines = (line.rstrip() for line in "".join(out).split("\n"))
    return "\n".join(line for line in lines if line)


def src_digest(d=None):
    """Digest of the code (comments and blank lines left out) of the sources
    that define and launch the single-box kernels: every csrc/ file but
    DIGEST_EXCLUDES, each with its name."""
    h = hashlib.sha256()
    d = d or os.path.join(ROOT, "paper_2509_18261_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f in DIGEST_EXCLUDES:
            continue
        h.update(f.encode() + b"\0" + code_of(open(os.path.join(d, f), encoding="utf-8").read()).encode() + b"\0")
    return h.hexdigest()[:16]


def profiled_row(kernel):
    """The row of `kernel` (bench name) in the committed one-kernel ncu
    capture on the 192^3 shrink, if it was taken on the current kernel
    sources: dict(fp64_per_unit, bytes_per_unit), else None."""
    path = os.path.join(ROOT, "profiles", "counters_c5_192.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"csrc_sha:\s*([0-9a-f]+)", txt)
    if not m or m.group(1) != src_digest():
        return None
    for line in txt.splitlines():
        cols = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cols) == 13 and cols[1] == kernel:
            return {"fp64_per_unit": float(cols[11]), "bytes_per_unit": float(cols[12]),
                    "dram_pct": float(cols[5]), "fp64_pipe_pct": float(cols[6]), "issue_pct": float(cols[7]),
                    "warps_active_pct": float(cols[8])}
    return None


def profiled_traffic(kernel, units):
    """DRAM bytes of one launch of `kernel` processing `units` (pairs or
    cells): the DRAM bytes per unit of the committed one-kernel ncu capture
    on the 192^3 shrink of the workload times `units`, if the capture was
    taken on the current kernel sources; else None.  (Traffic per pair is
    taken to scale with the pairs at equal particle density.)"""
    path = os.path.join(ROOT, "profiles", "counters_c5_192.md")
    if not os.path.exists(path) or not units:
        return None
    txt = open(path).read()
    m = re.search(r"csrc_sha:\s*([0-9a-f]+)", txt)
    if not m or m.group(1) != src_digest():
        return None
    for line in txt.splitlines():
        cols = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cols) == 13 and cols[1] == kernel:
            return float(cols[12]) * units
    return None


def measure_fp64_and_atomics():
    """FP64 fused-multiply-add and FP64 atomicAdd rates of this GPU, measured
    with the library's probe kernels (CUDA events on the launching stream,
    best of 5 after 3 warm-up launches)."""
    import torch

    from paper_2509_18261_gb300 import pmp

    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    threads, chains = pmp.pmp_probe_threads(), pmp.pmp_probe_chains()

    def best(fn, reps=5, warm=3):
        for _ in range(warm):
            fn()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return min(ts)

    out = {}
    blocks, iters = sms * 8, 4096
    buf = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    ms = best(lambda: pmp.pmp_probe_fp64(buf, blocks, iters))
    fmas = blocks * threads * chains * iters
    out["fp64_tflops"] = 2.0 * fmas / (ms * 1e-3) / 1e12
    out["fp64_dfma_per_clk_per_sm"] = None
    out["fp64_probe"] = (f"{blocks} blocks x {threads} threads x {chains} chains x {iters} DFMA "
                         f"(2 flops each), best of 5: {ms:.3f} ms")
    del buf
    for name, n_targets in (("atomic_l2_per_s", 1 << 20), ("atomic_hbm_per_s", 1 << 28)):
        tgt = torch.zeros(n_targets, dtype=torch.float64, device="cuda")
        n_adds = 1 << 28
        ms = best(lambda: pmp.pmp_probe_atomic(tgt, n_adds, sms * 16))
        out[name] = n_adds / (ms * 1e-3)
        del tgt
    out["atomic_probe"] = ("2^28 FP64 atomicAdd scattered over 2^20 doubles (8 MB, L2-resident) and over "
                           "2^28 doubles (2 GB), best of 5")
    torch.cuda.empty_cache()
    return out


def alg_bytes_fb(stage, n_fb, pairs, touched_state, touched_buf):
    """Algorithmic bytes of one launch of the supernova plan + gather or
    deposit kernel.  plan_gather: the particles read once (64 B), their 12
    gathered rows written (96 B), every touched state cell read once (40 B)
    and the plan written (8 B per pair).  deposit: positions and the six rows
    it uses read (72 B per particle), the plan read (8 B per pair), every
    touched state cell read once (40 B) and every touched buffer cell read
    and written once (80 B)."""
    if stage == "plan_gather":
        return 160 * n_fb + 8 * pairs + 40 * touched_state
    return 72 * n_fb + 8 * pairs + 40 * touched_state + 80 * touched_buf


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def gpu_local_cpus(local):
    """CPUs of the NUMA node the GPU hangs off (sysfs local_cpulist of its
    PCI function), or None.  Pinned host buffers allocated by a thread on
    those CPUs are placed in that node's memory."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(local), "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=30).stdout.strip().lower()
        if not out:
            return None
        dom, rest = out.split(":", 1)
        bdf = f"{int(dom, 16) & 0xffff:04x}:{rest}"
        spec = open(f"/sys/bus/pci/devices/{bdf}/local_cpulist").read().strip()
        cpus = set()
        for part in spec.split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        return cpus or None
    except Exception:
        return None


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import __graft_entry__

    # keep the host side (and the pinned buffers of the end-to-end leg) next
    # to the GPU's memory controller
    cpus = gpu_local_cpus(local)
    if cpus:
        try:
            os.sched_setaffinity(0, cpus & os.sched_getaffinity(0) or cpus)
        except OSError:
            pass
    __graft_entry__.build()
    from paper_2509_18261_gb300 import pmp
    from paper_2509_18261_gb300 import synthetic as syn

    if args.n:
        full = syn.WORKLOADS[args.workload]["n"]
        w = syn.make_workload(args.workload, n=args.n, count_scale=(args.n / full) ** 3,
                              keep_cluster_size=args.keep_cluster_size)
    else:
        w = syn.make_workload(args.workload)
    box = w["box"]
    dev = "cuda"
    state = torch.from_numpy(w["state"]).to(dev)
    fb = pmp.parts_to_device(w["fb"], dev)
    sk = pmp.parts_to_device(w["sink"], dev)
    n_fb, n_sk = fb["x"].numel(), sk["x"].numel()
    n_particles = n_fb + n_sk
    P_fb = pmp.Pass(w["fb_params"], box, state, fb, mode=args.mode)
    P_sk = pmp.Pass(w["sink_params"], box, state, sk, mode=args.mode)
    stream = torch.cuda.current_stream()

    phases = ["fb_zero", "fb_gather_deposit", "fb_fold", "fb_apply",
              "sink_zero", "sink_gather_deposit", "sink_fold", "sink_apply"]
    # own kernels per step (the CUB sorts, scans and run encoding are library
    # kernels).  ATOMIC: supernova pass zero, prologue, plan + gather,
    # deposit, fold, apply = 6; sink pass zero, prologue, per-cell records,
    # plan + gather + deposit, spread, fold, eta + apply, Step-4 return = 8.
    # SORTED: the pair counts in index order, pair values (with the sort's
    # lists), run and long-run kernels in place of the deposit (supernovae
    # 9); sinks plan, gather, the same four, no spread (12).  ROUNDED: a
    # deposit and a rounding kernel per pass (7 + 10).
    launches_per_step = {"atomic": 14, "sorted": 21, "rounded": 17}[args.mode]
    state0 = state.clone()
    sink0 = {k: sk[k].clone() for k in ("m", "px", "py", "pz")}

    def restore():
        state.copy_(state0)
        for k in sink0:
            sk[k].copy_(sink0[k])

    def cycle(events=None, restore_state=True):
        marks = []
        if restore_state:
            restore()

        def mark():
            if events is not None:
                e = torch.cuda.Event(enable_timing=True)
                e.record(stream)
                marks.append(e)

        for ps, parts in ((P_fb, fb), (P_sk, sk)):
            c = ps.ctx
            mark()
            pmp.pmp_zero_buffer(c, ps.buffer)
            mark()
            pmp.pmp_gather_deposit(c, ps.state, parts, ps.gathered, ps.buffer, args.mode, ps.workspace)
            mark()
            pmp.pmp_fold_ghosts(c, ps.buffer)
            mark()
            pmp.pmp_apply_limited(c, ps.state, ps.buffer, parts, ps.gathered, None, ps.workspace)
            mark()
        if events is not None:
            events.append(marks)

    for _ in range(args.warmup):
        cycle()
    torch.cuda.synchronize()
    for ps in (P_fb, P_sk):
        code, idx = pmp.pmp_get_error(ps.ctx)
        if code:
            raise RuntimeError(f"device error {code} at {idx}")

    for ps in (P_fb, P_sk):
        pmp.pmp_timing_read(ps.ctx)
        pmp.pmp_timing_enable(ps.ctx, True)
    clocks = Clocks(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    events = []
    t0.record(stream)
    for _ in range(args.steps):
        cycle(events)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms_total = t0.elapsed_time(t1)
    ms_per_step = max_over_ranks(world, ms_total / args.steps)
    phase_ms = {}
    for marks in events:
        # marks per pass: zero|gather+deposit|fold|apply boundaries (5 marks each)
        for p in range(2):
            m = marks[p * 5:(p + 1) * 5]
            for i in range(4):
                name = phases[p * 4 + i]
                phase_ms[name] = phase_ms.get(name, 0.0) + m[i].elapsed_time(m[i + 1]) / args.steps
    kernel_ms = {}
    for tag, ps in (("fb", P_fb), ("sink", P_sk)):
        for name, (nl, ms) in pmp.pmp_timing_read(ps.ctx).items():
            kernel_ms[f"{tag}_{name}"] = (nl / args.steps, ms / nl)
        pmp.pmp_timing_enable(ps.ctx, False)
    lim_fb = pmp.pmp_limiter_counts(P_fb.ctx)
    lim_sk = pmp.pmp_limiter_counts(P_sk.ctx)

    creation = sink_creation(P_sk, stream)

    # e2e: pinned host inputs -> device -> cycle -> results back to pinned host,
    # every step, through the public calls
    e2e = end_to_end(args, w, world, state, fb, sk, P_fb, P_sk, cycle, stream)

    # roofline of the dominant kernel (per-launch time from the library's
    # CUDA events on the launching stream)
    pairs = {"fb": kernel_cell_count(fb, box.n, w["fb_params"]["r_K"]),
             "sink": kernel_cell_count(sk, box.n, w["sink_params"]["r_K"])}
    hbm_peak, peak_src = peaks()
    step_ms_by_kernel = {k: nl * ms for k, (nl, ms) in kernel_ms.items()}
    by_time = sorted(step_ms_by_kernel, key=step_ms_by_kernel.get, reverse=True)
    dominant = by_time[0]
    measured = measure_fp64_and_atomics()

    def kernel_roof(name):
        r = roofline(name, kernel_ms[name][1], pairs, box, n_fb, n_sk, hbm_peak, peak_src)
        if r["bound"] == "alu" and r["unit"] == "TFLOP/s":
            r["peak_measured"] = measured["fp64_tflops"]
            r["frac_measured"] = r["achieved"] / measured["fp64_tflops"]
            r["peak_measured_source"] = "FP64 DFMA probe on this GPU, same run (pmp_probe_fp64)"
            row = profiled_row(name)
            kind = name.split("_", 1)[0]
            if row:
                # what binds it: the one-kernel counters of the 192^3 capture
                r["counters_192"] = {k: row[k] for k in ("issue_pct", "fp64_pipe_pct", "dram_pct",
                                                         "warps_active_pct")}
            if row and pairs.get(kind):
                # issued FP64 lane-operations (ncu, 192^3) over the FP64 issue peak (a DFMA = 2 flops)
                rate = row["fp64_per_unit"] * pairs[kind] / (kernel_ms[name][1] * 1e-3) / 1e12
                r["fp64_issue"] = {"lane_ops_per_pair": row["fp64_per_unit"], "T_lane_ops_per_s": rate,
                                   "peak": measured["fp64_tflops"] / 2.0,
                                   "frac": rate / (measured["fp64_tflops"] / 2.0)}
        return r

    roof = kernel_roof(dominant)
    if dominant in ("fb_plan_gather", "fb_deposit"):
        # the same launch seen as an HBM kernel: algorithmic bytes over time
        touched = touched_cells(P_fb, w["fb_params"], box, state0, fb)
        ab = alg_bytes_fb(dominant.split("_", 1)[1], n_fb, pairs["fb"], touched["state"], touched["buffer"])
        gbs = ab / (kernel_ms[dominant][1] * 1e-3) / 1e9
        roof["hbm_view"] = {"algorithmic_bytes": ab, "GB/s": gbs, "frac": gbs / hbm_peak,
                            "touched_cells": touched}
        if roof.get("traffic"):
            roof["traffic_ratio"] = roof["traffic"] / ab
    # the same for the next two kernels by time per step
    roof["others"] = [kernel_roof(k) for k in by_time[1:3]]

    hbm_passes = cell_pass_hbm(kernel_ms, box, hbm_peak)

    result = {
        "metric": METRIC,
        "value": n_particles * world / (ms_per_step * 1e-3),
        "unit": "particles/s",
        "cells_per_s": box.ncells_valid * world / (ms_per_step * 1e-3),
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {
            "workload": (f"{args.workload}: {box.n[0]}^3 box, {box.g} ghost cells, 5 FP64 fields; "
                         f"{n_fb} supernova particles (r_K=2, S=4) + {n_sk} sinks (r_K=4), "
                         "25% in 256 Plummer clusters (a=2 cells); supernova pass then sink pass"),
            "mode": args.mode,
            "l2": f"inputs larger than L2 (state + buffer {2 * 8 * 5 * box.ncells_padded / 1e9:.1f} GB)",
            "parallelism": f"replicas x{world}",
            "kernel_pairs": pairs,
        },
        "phases_ms": {k: round(v, 4) for k, v in phase_ms.items()},
        "kernels_ms_per_launch": {k: round(v[1], 4) for k, v in sorted(kernel_ms.items())},
        "limiter": {"fb_cells_eta_lt_1": lim_fb[0], "fb_noroot": lim_fb[1], "sink_cells_eta_lt_1": lim_sk[0]},
        "roofline": roof,
        "measured_peaks": measured,
        "hbm_passes": hbm_passes,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "host_affinity": (f"{len(cpus)} CPUs local to the GPU" if cpus else "unchanged"),
    }
    result["sink_creation_c5_512"] = creation
    result["pm_deposit_c5_512"] = pm_deposit(args, w, state, fb, stream)
    result["fwd_bwd_c4_128"] = fwd_bwd(args)
    if not args.no_batched:
        result["batched_c3"] = batched(args)
        result["deposit_modes_c2_256"] = deposit_modes(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(result), flush=True)


def end_to_end(args, w, world, state, fb, sk, P_fb, P_sk, cycle, stream):
    """The cycle measured from pinned host memory to pinned host memory: every
    step copies its inputs (gas state, both particle sets) to the device, runs
    the two passes and copies the results (gas state, sink masses and
    momenta) back.  Pipelined over three device input sets: the copies of
    step k+1 (in) and k-1 (out) run while step k computes, each direction
    split over --copy-streams copy streams, each copy ordered after the work
    it depends on by events.  Also reported: the same steps run one after another on one
    stream (serial_ms_per_step)."""
    import torch

    from paper_2509_18261_gb300 import pmp

    h_state = torch.from_numpy(w["state"]).pin_memory()
    h_fb = {k: torch.from_numpy(v).pin_memory() for k, v in w["fb"].items()}
    h_sk = {k: torch.from_numpy(v).pin_memory() for k, v in w["sink"].items()}
    NSETS = 3  # device input sets of the pipelined form (below)
    outs = [dict(state=torch.empty_like(h_state).pin_memory(),
                 sk={k: torch.empty_like(h_sk[k]).pin_memory() for k in ("m", "px", "py", "pz")})
            for _ in range(NSETS)]
    bi = h_state.numel() * 8 + sum(v.numel() * 8 for v in h_fb.values()) + sum(v.numel() * 8 for v in h_sk.values())
    bo = h_state.numel() * 8 + sum(v.numel() * 8 for v in outs[0]["sk"].values())
    steps = max(args.e2e_steps if args.e2e_steps else args.steps, 2)

    def copy_in(st, f, k_):
        st.copy_(h_state, non_blocking=True)
        for k in h_fb:
            f[k].copy_(h_fb[k], non_blocking=True)
        for k in h_sk:
            k_[k].copy_(h_sk[k], non_blocking=True)

    def copy_out(o, st, k_):
        o["state"].copy_(st, non_blocking=True)
        for k in o["sk"]:
            o["sk"][k].copy_(k_[k], non_blocking=True)

    def run_passes(ps):
        for P, parts in ps:
            c = P.ctx
            pmp.pmp_zero_buffer(c, P.buffer)
            pmp.pmp_gather_deposit(c, P.state, parts, P.gathered, P.buffer, args.mode, P.workspace)
            pmp.pmp_fold_ghosts(c, P.buffer)
            pmp.pmp_apply_limited(c, P.state, P.buffer, parts, P.gathered, None, P.workspace)

    # serial: copy in, cycle, copy out, all on the compute stream
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        copy_in(state, fb, sk)
        run_passes(((P_fb, fb), (P_sk, sk)))
        copy_out(outs[0], state, sk)
    e1.record(stream)
    torch.cuda.synchronize()
    serial_ms = max_over_ranks(world, e0.elapsed_time(e1) / steps)

    # pipelined over NSETS device input sets, each with its own passes: the
    # copy of step k+1's inputs (in) and of step k-1's results (out) run
    # while step k computes; with three sets an in-copy never waits for the
    # out-copy of the same set (two sets chain the two copies of every step
    # one after the other)
    mode = args.mode
    sets = [(state, fb, sk, ((P_fb, fb), (P_sk, sk)))]
    extra = []
    for _ in range(NSETS - 1):
        st1 = torch.empty_like(state)
        fb1 = {k: torch.empty_like(v) for k, v in fb.items()}
        sk1 = {k: torch.empty_like(v) for k, v in sk.items()}
        Q_fb = pmp.Pass(w["fb_params"], P_fb.box, st1, fb1, mode=mode)
        Q_sk = pmp.Pass(w["sink_params"], P_sk.box, st1, sk1, mode=mode)
        extra += [Q_fb, Q_sk]
        sets.append((st1, fb1, sk1, ((Q_fb, fb1), (Q_sk, sk1))))
    # each direction's copies are split over NCOPY streams (a single copy
    # moves at the rate of one copy engine)
    NCOPY = max(1, args.copy_streams)
    s_in = [torch.cuda.Stream() for _ in range(NCOPY)]
    s_out = [torch.cuda.Stream() for _ in range(NCOPY)]

    def pieces(t):
        flat = t.view(-1)
        n = flat.numel()
        step = (n + NCOPY - 1) // NCOPY
        return [flat[i * step:min(n, (i + 1) * step)] for i in range(NCOPY)]

    h_pieces = pieces(h_state)
    o_pieces = [pieces(o["state"]) for o in outs]
    d_pieces = [pieces(st_[0]) for st_ in sets]

    def copy_in_split(j, after):
        evs = []
        for i, s_ in enumerate(s_in):
            with torch.cuda.stream(s_):
                for e in after:
                    s_.wait_event(e)
                d_pieces[j][i].copy_(h_pieces[i], non_blocking=True)
                if i == 0:
                    for k in h_fb:
                        sets[j][1][k].copy_(h_fb[k], non_blocking=True)
                    for k in h_sk:
                        sets[j][2][k].copy_(h_sk[k], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(s_)
                evs.append(ev)
        return evs

    def copy_out_split(i_, after):
        evs = []
        for i, s_ in enumerate(s_out):
            with torch.cuda.stream(s_):
                s_.wait_event(after)
                o_pieces[i_][i].copy_(d_pieces[i_][i], non_blocking=True)
                if i == 0:
                    for k in outs[i_]["sk"]:
                        outs[i_]["sk"][k].copy_(sets[i_][2][k], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(s_)
                evs.append(ev)
        return evs

    ev_in = [[] for _ in range(NSETS)]
    ev_out = [[] for _ in range(NSETS)]
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ev_in[0] = copy_in_split(0, [e0])
    for k in range(steps):
        i, j = k % NSETS, (k + 1) % NSETS
        if k + 1 < steps:
            # set j's results of an earlier step have left the device
            ev_in[j] = copy_in_split(j, ev_out[j])
        for e in ev_in[i]:
            stream.wait_event(e)
        run_passes(sets[i][3])
        done = torch.cuda.Event()
        done.record(stream)
        ev_out[i] = copy_out_split(i, done)
    for i in range(NSETS):
        for e in ev_out[i]:
            stream.wait_event(e)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(world, e0.elapsed_time(e1) / steps)
    for P in extra:
        code, idx = pmp.pmp_get_error(P.ctx)
        if code:
            raise RuntimeError(f"e2e: device error {code} at {idx}")
        P.ctx.close()
    n_particles = sum(v.numel() for v in (fb["x"], sk["x"]))
    return {"value": n_particles * world / (ms * 1e-3), "unit": "particles/s", "ms_per_step": ms,
            "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "steps": steps,
            "serial_ms_per_step": serial_ms,
            "overlap": f"three device input sets: the copies of step k+1 (in) and k-1 (out) run during step k, each "
                       f"direction split over {NCOPY} copy streams"}


def touched_cells(P_fb, params, box, state0, fb):
    """Distinct buffer cells (ghosts included) and distinct state cells that
    one supernova deposit touches: a deposit on the initial state, counted
    from the buffer's density row before and after the fold."""
    import torch

    from paper_2509_18261_gb300 import pmp

    ps = P_fb
    ps.state.data.copy_(state0)
    pmp.pmp_zero_buffer(ps.ctx, ps.buffer)
    pmp.pmp_gather_deposit(ps.ctx, ps.state, fb, ps.gathered, ps.buffer, ps.mode, ps.workspace)
    rho = ps.buffer.data[0, :box.ncells_padded]
    tb = int(torch.count_nonzero(rho).item())
    pmp.pmp_fold_ghosts(ps.ctx, ps.buffer)
    g = box.g
    px, py, pz = box.padded
    v = ps.buffer.data[0, :box.ncells_padded].reshape(pz, py, px)[g:pz - g, g:py - g, g:px - g]
    ts = int(torch.count_nonzero(v).item())
    torch.cuda.synchronize()
    return {"buffer": tb, "state": ts}


def sink_creation(P_sk, stream):
    """Sink creation (Sec. 3.1.2) on the 512^3 state right after the timed
    cycles, with the last sink pass's summed buffer: CUDA-event time of one
    pmp_create_sinks (flags, scan, creation) and the number of new sinks."""
    import torch

    from paper_2509_18261_gb300 import pmp

    ws = torch.empty(pmp.pmp_create_sinks_workspace_size(P_sk.ctx, P_sk.state), dtype=torch.uint8, device="cuda")
    cap = 1 << 20
    out = {k: torch.empty(cap, dtype=torch.float64, device="cuda") for k in ("x", "y", "z", "m", "px", "py", "pz")}
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    pmp.pmp_create_sinks(P_sk.ctx, P_sk.state, P_sk.buffer, out, cnt, ws)
    e1.record(stream)
    torch.cuda.synchronize()
    code, idx = pmp.pmp_get_error(P_sk.ctx)
    if code:
        raise RuntimeError(f"sink creation: device error {code} at {idx}")
    n = int(cnt.item())
    return {"ms": e0.elapsed_time(e1), "new_sinks": n,
            "new_mass": float(out["m"][:min(n, cap)].sum().item()) if n else 0.0,
            "cells_per_s": P_sk.box.ncells_valid / (e0.elapsed_time(e1) * 1e-3)}


def pm_deposit(args, w, state, fb, stream):
    """The particle-mesh (PM/PIC) subset of the cycle, Steps 1, 2 and 5 of
    Sec. 2.2: the 14,680,064 supernova particles of the 512^3 workload
    deposited as mass, momentum and energy with the supernova kernel (r_K = 2,
    S = 4) and added to the state without a limiter.  CUDA-event time of one
    pass, mean over `steps` after 3 warm-ups (the state keeps accumulating;
    the work per pass is the same)."""
    import torch

    from paper_2509_18261_gb300 import pmp
    from paper_2509_18261_gb300 import synthetic as syn

    P = pmp.Pass(syn.mass_params(), w["box"], state, fb, mode=args.mode)
    times = []
    for it in range(3 + max(args.steps, 1)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P.run()
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= 3:
            times.append(e0.elapsed_time(e1))
    code, idx = pmp.pmp_get_error(P.ctx)
    if code:
        raise RuntimeError(f"pm deposit: device error {code} at {idx}")
    P.ctx.close()
    ms = sum(times) / len(times)
    n = fb["x"].numel()
    return {"ms_per_pass": ms, "particles_per_s": n / (ms * 1e-3),
            "cells_per_s": w["box"].ncells_valid / (ms * 1e-3), "particles": n, "mode": args.mode}


def fwd_bwd(args):
    """Forward + backward of one supernova pass on the 128^3 workload (262,144
    supernovae, half in 32 clusters): CUDA-event times of the forward (gather,
    deposit, fold, limited apply) and of pmp_backward, after 3 warm-ups."""
    import torch

    from paper_2509_18261_gb300 import pmp
    from paper_2509_18261_gb300 import synthetic as syn

    w = syn.make_workload("c4_128")
    box = w["box"]
    u0 = torch.from_numpy(w["state"]).cuda()
    u = u0.clone()
    parts = pmp.parts_to_device(w["fb"])
    n = parts["x"].numel()
    ps = pmp.Pass(w["fb_params"], box, u, parts, mode="atomic")
    rng = torch.Generator(device="cuda").manual_seed(4)
    gU = torch.randn(u.shape, dtype=torch.float64, device="cuda", generator=rng)
    g = torch.empty((8, n), dtype=torch.float64, device="cuda")
    state_in = pmp.Mesh(u0, box.n, box.g)
    stream = torch.cuda.current_stream()
    f_ms, b_ms = [], []
    for it in range(3 + max(args.steps, 1)):
        u.copy_(u0)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        ps.run()
        e1.record(stream)
        pmp.pmp_backward(ps.ctx, state_in, ps.buffer, parts, ps.gathered_view(), gU, g, ps.workspace)
        e2.record(stream)
        torch.cuda.synchronize()
        if it >= 3:
            f_ms.append(e0.elapsed_time(e1))
            b_ms.append(e1.elapsed_time(e2))
    code, idx = pmp.pmp_get_error(ps.ctx)
    if code:
        raise RuntimeError(f"device error {code} at {idx}")
    ps.ctx.close()
    fm, bm = sum(f_ms) / len(f_ms), sum(b_ms) / len(b_ms)
    return {"fwd_ms": fm, "bwd_ms": bm, "total_ms": fm + bm, "particles": n,
            "workload": "c4_128: 128^3, 4 ghosts, 262,144 supernovae (half in 32 Plummer clusters)"}


def deposit_modes(args):
    """Step 1 on the 256^3 workload (1,048,576 supernovae, half in 32 Plummer
    clusters) in the three accumulation modes: CUDA-event time of pmp_deposit
    (ATOMIC; SORTED with its pair sort; ROUNDED with its error bound and the
    rounding pass of App. A.1), mean of `steps` calls after 3 warm-ups.  Then
    the reproducibility of each mode: buffer values (of cells some particle
    reaches) that differ between two runs on the same input, and between the
    input and the same particles in a seeded random order."""
    import torch

    from paper_2509_18261_gb300 import pmp
    from paper_2509_18261_gb300 import synthetic as syn

    w = syn.make_workload("c2_256")
    box = w["box"]
    st = torch.from_numpy(w["state"]).cuda()
    parts = pmp.parts_to_device(w["fb"])
    n = parts["x"].numel()
    gen = torch.Generator(device="cuda").manual_seed(2509)
    perm = torch.randperm(n, device="cuda", generator=gen)
    parts2 = {k: v[perm].contiguous() for k, v in parts.items()}
    stream = torch.cuda.current_stream()
    out = {"workload": "c2_256: 256^3, 4 ghosts, 1,048,576 supernovae (half in 32 Plummer clusters), Step 1 only",
           "ms": {}, "differing_values_between_orders": {}}
    touched = None
    out["differing_values_between_runs"] = {}
    for mode, M in (("atomic", None), ("sorted", None), ("rounded", 28), ("rounded", 16), ("rounded", 8)):
        bufs = []
        for pp, timed in ((parts, M in (None, 28)), (parts, False), (parts2, False)):
            ps = pmp.Pass(w["fb_params"], box, st, pp, mode=mode)
            if M is not None:
                pmp.pmp_set_rounding_margin(ps.ctx, M)
            c = ps.ctx
            pmp.pmp_gather(c, ps.state, pp, ps.gathered, mode, ps.workspace)
            if timed:
                pmp.pmp_timing_read(c)
                pmp.pmp_timing_enable(c, True)
            times = []
            for it in range(3 + (max(args.steps, 1) if timed else 0)):
                pmp.pmp_zero_buffer(c, ps.buffer)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pmp.pmp_deposit(c, ps.state, pp, ps.gathered, ps.buffer, mode, ps.workspace)
                e1.record(stream)
                torch.cuda.synchronize()
                if it >= 3:
                    times.append(e0.elapsed_time(e1))
            code, idx = pmp.pmp_get_error(c)
            if code:
                raise RuntimeError(f"deposit modes: device error {code} at {idx}")
            if times:
                out["ms"][mode] = sum(times) / len(times)
                stages = pmp.pmp_timing_read(c)
                pmp.pmp_timing_enable(c, False)
                out.setdefault("stage_ms", {})[mode] = {k: round(ms / nl, 4) for k, (nl, ms) in stages.items()}
            bufs.append(ps.buffer.data.clone())
            c.close()
        a, a2, b = bufs
        if touched is None:
            touched = a != 0
        key = mode if M is None else f"rounded_M{M}"
        out["differing_values_between_runs"][key] = int(((a.view(torch.int64) != a2.view(torch.int64)) & touched)
                                                        .sum().item())
        out["differing_values_between_orders"][key] = int(((a.view(torch.int64) != b.view(torch.int64)) & touched)
                                                          .sum().item())
    out["touched_values"] = int(touched.sum().item())
    out["full_cycle"] = c2_full_cycle(args, w, st, parts)
    return out


def c2_full_cycle(args, w, st0, parts):
    """One whole supernova pass on the 256^3 workload -- zero, gather +
    deposit, fold, limited apply -- in the ATOMIC and SORTED modes: CUDA-event
    time per pass (mean of `steps` passes after 3 warm-ups, each from the
    initial state), particles/s and cells/s."""
    import torch

    from paper_2509_18261_gb300 import pmp

    box = w["box"]
    stream = torch.cuda.current_stream()
    out = {}
    n = parts["x"].numel()
    for mode in ("atomic", "sorted"):
        st = st0.clone()
        ps = pmp.Pass(w["fb_params"], box, st, parts, mode=mode)
        times = []
        for it in range(3 + max(args.steps, 1)):
            st.copy_(st0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ps.run()
            e1.record(stream)
            torch.cuda.synchronize()
            if it >= 3:
                times.append(e0.elapsed_time(e1))
        code, idx = pmp.pmp_get_error(ps.ctx)
        if code:
            raise RuntimeError(f"c2 full cycle: device error {code} at {idx}")
        ms = sum(times) / len(times)
        out[mode] = {"ms": ms, "particles_per_s": n / (ms * 1e-3), "cells_per_s": box.ncells_valid / (ms * 1e-3)}
        ps.ctx.close()
        del ps, st
    torch.cuda.empty_cache()
    return out


def batched_hbm_view(nvalid, npadded, ms_per_cycle, hbm_peak, peak_src):
    """HBM view of one batched mixed cycle (two passes) from the per-unit
    algorithmic bytes of the single-box passes: per pass, zero 40 B per buffer
    cell, fold 120 B per ghost-shell cell, apply 120 B per valid cell.  The
    particle terms (gather, deposit and Step 4 over a few thousand particles)
    are under 1% and left out.  The fused fold + update reads and writes the
    state only where the summed change is non-zero, so the DRAM bytes it moves
    are below this figure."""
    per_pass = 40 * npadded + 120 * (npadded - nvalid) + 120 * nvalid
    alg = 2 * per_pass
    gbs = alg / (ms_per_cycle * 1e-3) / 1e9
    return {"algorithmic_bytes_per_cycle": alg, "GB/s": gbs, "peak": hbm_peak, "frac": gbs / hbm_peak,
            "peak_source": peak_src,
            "bytes": "per pass: zero 40 B per buffer cell, fold 120 B per ghost-shell cell, apply 120 B per valid cell"}


def batched(args):
    """The batched form on the 512-patch workload (8x8x8 periodic super-grid,
    edges from {16,24,32,48,64} per axis, power-law particle counts, 1/8
    sinks): one mixed cycle (supernova pass, then sink pass) per step with the
    autotuned per-bin strategies, run as one persistent launch per pass, as
    that launch replayed from a CUDA graph, and as the plain per-patch launch
    loop.  CUDA-event times of the two passes (the state restore before each
    step is outside them), mean over `steps` after 3 warm-ups."""
    import torch

    from paper_2509_18261_gb300 import pmp
    from paper_2509_18261_gb300 import synthetic as syn

    w = syn.make_batch_workload()
    batch = w["batch"]
    st0 = torch.from_numpy(w["state"]).cuda()
    st = st0.clone()
    fb = pmp.parts_to_device(w["fb"])
    sk = pmp.parts_to_device(w["sink"])
    sk0 = {k: sk[k].clone() for k in ("m", "px", "py", "pz")}
    passes = [pmp.BatchPass(w["fb_params"], batch, st, fb, w["fb_first"]),
              pmp.BatchPass(w["sink_params"], batch, st, sk, w["sink_first"])]
    chosen = []
    for bp in passes:
        chosen.append(pmp.pmp_batch_autotune(bp.h, st, bp.buffer, bp.parts, bp.gathered, deterministic=True))
    stream = torch.cuda.current_stream()

    def restore():
        st.copy_(st0)
        for k in sk0:
            sk[k].copy_(sk0[k])

    out = {}
    for launch in ("persistent", "graph", "per_patch"):
        times = []
        for it in range(3 + max(args.steps, 1)):
            restore()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for bp in passes:
                bp.run(launch)
            e1.record(stream)
            torch.cuda.synchronize()
            if it >= 3:
                times.append(e0.elapsed_time(e1))
        out[launch] = sum(times) / len(times)
    for bp in passes:
        code, idx = pmp.pmp_get_error(bp.ctx)
        if code:
            raise RuntimeError(f"batched: device error {code} at {idx}")
    grid, items = pmp.pmp_batch_info(passes[0].h)
    for bp in passes:
        bp.close()
    n_particles = int(w["fb_first"][-1] + w["sink_first"][-1])
    best = min(out["persistent"], out["graph"])
    hbm_peak, peak_src = peaks()
    return {
        "ms_per_cycle": {k: round(v, 4) for k, v in out.items()},
        "hbm_view": batched_hbm_view(batch.ncells_valid, batch.ncells_padded, best, hbm_peak, peak_src),
        "speedup_vs_per_patch": out["per_patch"] / best,
        "cells_per_s": batch.ncells_valid / (best * 1e-3),
        "particles_per_s": n_particles / (best * 1e-3),
        "strategy_per_bin": {"fb": chosen[0], "sink": chosen[1]},
        "persistent_grid": grid,
        "workload": (f"c3_batched: {batch.np} patches on an 8x8x8 periodic super-grid, {batch.ncells_valid} valid "
                     f"cells, {int(w['fb_first'][-1])} supernovae + {int(w['sink_first'][-1])} sinks, 4 ghosts"),
    }


# ---------------------------------------------------------------------------
# CPU oracle: the baseline leg and the reference arm
# ---------------------------------------------------------------------------

def oracle_cycle_sample(n, seed_workload=WORKLOAD):
    """One mixed cycle of the oracle on the workload shrunk to an n^3 box with
    the same particle density; returns (seconds, particles, cells)."""
    import oracle
    from paper_2509_18261_gb300 import synthetic as syn

    full = syn.WORKLOADS[seed_workload]["n"]
    w = syn.make_workload(seed_workload, n=n, count_scale=(n / full) ** 3)
    box = w["box"]
    st = w["state"].copy()
    t = time.perf_counter()
    oracle.cycle(w["fb_params"], box, st, w["fb"])
    oracle.cycle(w["sink_params"], box, st, w["sink"])
    dt = time.perf_counter() - t
    return dt, len(w["fb"]["x"]) + len(w["sink"]["x"]), box.ncells_valid


def cpu_baseline(args):
    dt, npart, ncells = oracle_cycle_sample(args.cpu_sample_n)
    return {"value": npart / dt, "unit": "particles/s", "cores": 1, "host_cpus": os.cpu_count(), "kind": "oracle",
            "cells_per_s": ncells / dt,
            "sample": f"one mixed cycle of the same workload shrunk to {args.cpu_sample_n}^3 at equal particle "
                      f"density ({npart} particles), single-threaded C oracle, {dt:.2f} s"}


def run_reference(args, world, rank):
    if rank != 0:
        return
    n = 64
    for _ in range(args.warmup):
        oracle_cycle_sample(n)
    times = []
    npart = ncells = 0
    for _ in range(args.steps):
        dt, npart, ncells = oracle_cycle_sample(n)
        times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = npart / (ms * 1e-3)
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "particles/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload} shrunk to {n}^3 at equal particle density ({npart} particles)"},
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": 1, "host_cpus": os.cpu_count(), "kind": "oracle",
                         "sample": f"{n}^3 sample of {args.workload}, one mixed cycle per step"},
        "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        run_reference(args, world, rank)
        return
    world, rank, local = dist_init()
    run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
