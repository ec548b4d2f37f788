#!/usr/bin/env python
"""Throughput of the exponential-integrator step on GB300.

Workload: the 128^3 head phantom (per-voxel D with 10 % noise, D_w = 0.13,
D_g = 0.013 mm^2/day, rho = 0.025/day, h = 1 mm), 100 steps of tau = 7.3 days
(two years).  One bench step = one et_run of those 100 steps from u0 on data
resident in HBM; value = voxel-steps per second over all ranks (Mvoxel-steps/s).
Coefficient setup (et_set_coeffs) is timed separately.  N > 1 runs independent
replicas, one per GPU (weak scaling, no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (the method's plain definition)
on the host cores on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N_GRID = 128
NSTEPS = 100
TAU = 7.3
RHO = 0.025
NOISE = 0.1
METRIC = "exp-integrator Mvoxel-steps/s at 128^3 (plain vs chosen form), % HBM roofline"
UNIT = "Mvoxel-steps/s"
WORKLOAD = "128^3 head phantom, D noise 10%, rho 0.025/d, 100 steps x tau 7.3 d (2 years), zero-flux"
# Algorithmic bytes and flops per voxel of one Taylor-term launch (conservative
# operator).  Sub-step 0 is evaluated by Horner's rule: read z 8, write z 8,
# three face-weight fields 24, diagonal 8, residual 8 = 56 B (FP64 and DF64
# pairs; 28 B in FP32), 7 FMA + 1 MUL = 15 flops (DF64: the compensated 8-term
# dot product, 118 FP32 flops).  Terms of later sub-steps also read and write
# the running sum: 72 B (36 B), 17 flops (DF64 139).
HORNER_BYTES = {"f64": 56, "df64": 56, "f32": 28}
HORNER_FLOPS = {"f64": 15, "df64": 118, "f32": 15}
TERM_BYTES = {"f64": 72, "df64": 72, "f32": 36}
TERM_FLOPS = {"f64": 17, "df64": 139, "f32": 17}
# In warp rows without off-diagonal entries (D = 0 around them) the one-term
# FP64 and DF64 kernels evaluate dt z + beta b only: z, the diagonal and b in,
# z out (4 fields; 6 with the running sum), 1 MUL + 1 FMA = 3 flops (5 with
# the running sum; DF64 counts its pair arithmetic as 118 / 139 for every
# voxel, an upper bound).  The FP32 kernels evaluate every row.  The DF64
# two-term kernel skips the arithmetic of such voxels, but its TMA boxes still
# bring every field of its tiles, so its bytes are those of every row.
ZERO_ROW_FIELDS = {"horner": 4, "term": 6}
ZERO_ROW_FLOPS = {"horner": 3, "term": 5}
# the kernels whose loads skip those rows: whether their flops do too
ZERO_ROW_KERNELS = {"term_kernel_f64": True, "term_kernel_df64": True,
                    "batch_term_f64_kernel": True, "batch_term_df64_kernel": True}


def launch_mix(prec, s, m, pairs, zero_frac=0.0, zero_flops=True):
    """(launches, algorithmic bytes, flops) per voxel of one step's term chain.

    Sub-step 0 has m - 1 Horner terms, each later sub-step m terms.  With pairs
    (the DF64 default) two consecutive terms of a sub-step share one launch
    that reads z, the weights, the diagonal and b once and writes one z (and the
    sum), so a pair moves the bytes of one single term and does twice its flops.
    zero_frac: the share of voxels in warp rows without off-diagonal entries,
    whose terms move the bytes of 4 (6) fields; zero_flops: their flops are
    those of dt z + beta b too (else every product is evaluated)."""
    def count(nterms):
        return (nterms // 2, nterms % 2) if pairs else (0, nterms)
    ph, sh = count(m - 1)
    pt, st = count(m)
    launches = ph + sh + (s - 1) * (pt + st)
    zb = VALUE_BYTES[prec]
    hb = (1 - zero_frac) * HORNER_BYTES[prec] + zero_frac * zb * ZERO_ROW_FIELDS["horner"]
    tb = (1 - zero_frac) * TERM_BYTES[prec] + zero_frac * zb * ZERO_ROW_FIELDS["term"]
    if prec == "df64" or not zero_flops:
        hf, tf = HORNER_FLOPS[prec], TERM_FLOPS[prec]
    else:
        hf = (1 - zero_frac) * HORNER_FLOPS[prec] + zero_frac * ZERO_ROW_FLOPS["horner"]
        tf = (1 - zero_frac) * TERM_FLOPS[prec] + zero_frac * ZERO_ROW_FLOPS["term"]
    nbytes = hb * (ph + sh) + tb * (s - 1) * (pt + st)
    flops = hf * (2 * ph + sh) + tf * (s - 1) * (2 * pt + st)
    return launches, nbytes, flops


# DRAM bytes per voxel of one term launch (dram__bytes_read.sum +
# dram__bytes_write.sum over the voxels of the launch) from one ncu capture of
# each kernel in its steady state (--cache-control none, a launch in the middle
# of a run; a two-term launch covers two terms), keyed by (form, kernel, grid
# edge or "batch"), with the SHA-256 prefix of the kernel's source file at the
# capture: a kernel changed since then reports null.  The batched launch is
# captured on the first 8 grids of the batch (19.0 M voxels) and scaled to the
# whole launch by its voxels (traffic grows with them: no re-reads across grids).
TERM_TRAFFIC = {
    ("f64", "term_kernel_f64", 128): (32060160 / 128 ** 3, "be16966deb22"),
    ("f32", "term_quad_kernel", 128): (403712 / 128 ** 3, "a6bae89026da"),
    ("df64", "term2_kernel", 128): (101615872 / 128 ** 3, "bac2a73d8148"),
    ("df64", "term2_kernel", 192): (415784704 / 192 ** 3, "bac2a73d8148"),
    ("f32", "term2_quad_kernel", 160): (101667584 / 160 ** 3, "4cf51af4dc30"),
    ("f32", "term2_quad_kernel", 192): (200058368 / 192 ** 3, "4cf51af4dc30"),
    ("f32", "batch_term2_quad_kernel", "batch"): (560926464 / 19017728, "4cf51af4dc30"),
}
KERNEL_SOURCE = {"term_kernel_f64": "et_kernels.cu", "term2_kernel": "et_fused.cu",
                 "term_quad_kernel": "et_quad.cu", "term_kernel_df64": "et_df64.cu",
                 "term2_quad_kernel": "et_quadpair.cu", "batch_term2_quad_kernel": "et_quadpair.cu"}


def source_sha(kernel):
    import hashlib
    path = os.path.join(ROOT, "paper_2402_02273_gb300", "csrc", KERNEL_SOURCE.get(kernel, ""))
    if not os.path.isfile(path):
        return None
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:12]


def term_traffic(prec, kernel, grid, voxels):
    """Steady-state DRAM bytes of one launch over `voxels` voxels, or None (no
    capture of this kernel as it stands at this size)."""
    entry = TERM_TRAFFIC.get((prec, kernel, grid))
    if not entry or entry[1] != source_sha(kernel):
        return None
    return entry[0] * voxels


def term_kernel_of(prec, single_terms, n):
    """The kernel that runs the Taylor terms of a single grid (the library's
    default choice): FP64 one term per launch; DF64 two per launch (TMA-fed);
    FP32 one per launch on the four-voxel kernel while the Horner chain's
    fields (28 B per voxel) stay within 0.75 L2 sizes, else two per launch on
    the four-voxel two-term kernel.  --single-terms: one everywhere."""
    if prec == "f64":
        return "term_kernel_f64", False
    if prec == "df64":
        return ("term_kernel_df64", False) if single_terms else ("term2_kernel", True)
    if single_terms or 28.0 * n <= 0.75 * L2_BYTES:
        return "term_quad_kernel", False
    return "term2_quad_kernel", True
L2_FLUSH_BYTES = 256 << 20
ADJ_STEPS = 50  # the adjoint workload: 128^3, 50 steps, checkpoints every 10
ADJ_CK = 10
BATCH_COUNT = 64  # the many-patient workload: 64 grids of {96..160}^3, 100 steps each


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=N_GRID)
    ap.add_argument("--nsteps", type=int, default=NSTEPS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip timing the adjoint form")
    ap.add_argument("--adjoint-forms", default="f64,f32")
    ap.add_argument("--no-forms", action="store_true", help="time the plain FP64 form only")
    ap.add_argument("--single-terms", action="store_true", help="one Taylor term per launch in every form")
    ap.add_argument("--every-row", action="store_true",
                    help="evaluate the stencil in every row (no zero-row skip) in every form")
    ap.add_argument("--every-row-forms", default="f64",
                    help="forms also timed on the 128^3 run with every row evaluated, for comparison")
    ap.add_argument("--no-batch", action="store_true", help="skip timing the batched many-grid form")
    ap.add_argument("--batch-count", type=int, default=BATCH_COUNT)
    ap.add_argument("--batch-runs", type=int, default=1, help="timed runs of the batched form (one warm-up run)")
    ap.add_argument("--batch-forms", default="f64,df64,f32")
    ap.add_argument("--forms", default="f64,df64,f32",
                    help="comma-separated precision forms to time (the first one is the headline)")
    ap.add_argument("--large-grid", type=int, default=192,
                    help="edge of the grid beyond the L2 on which the FP32 / DF64 forms are also timed (0: skip)")
    ap.add_argument("--large-forms", default="f32,df64")
    ap.add_argument("--no-cn", action="store_true", help="skip the Crank-Nicolson comparison line")
    ap.add_argument("--cn-rtol", type=float, default=1e-12)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value, device="cuda"):
    """The largest value over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, voxels, steps_per_run, ms_per_step):
    """Voxel-steps per second of all ranks together (replicas: each rank runs its own grid)."""
    return world * voxels * steps_per_run / (ms_per_step * 1e-3) / 1e6


def _oracle_rate(D, u0, seconds, theta=0.5, stop_tol=1e-18):
    """Steps of the oracle from u0 for about `seconds`; returns (Mvoxel-steps/s, steps, seconds)."""
    import oracle
    P = oracle.Problem(D, rho=RHO)
    u = u0.copy()
    steps = 0
    t0 = time.perf_counter()
    while steps < NSTEPS:
        u, _ = P.run(u, TAU, 1, theta=theta, stop_tol=stop_tol)
        steps += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return D.size * steps / dt / 1e6, steps, dt


def cpu_baseline(D, u0, seconds=12.0, extra_seconds=6.0):
    """The FP64 oracle as it stands, on the host cores, on the first steps of the run.

    The headline is all cores with the oracle's own tight schedule (theta 0.5,
    tail bound 1e-18).  `variants` adds one core, and a baseline mode whose
    schedule is as loose as the GPU's (theta 6.4, the GPU's sub-step size at
    this workload, tail bound 1e-13)."""
    import oracle
    cores = oracle.get_threads()
    value, steps, dt = _oracle_rate(D, u0, seconds)
    variants = {}
    oracle.set_threads(1)
    try:
        v1, s1, t1 = _oracle_rate(D, u0, extra_seconds)
    finally:
        oracle.set_threads(cores)
    variants["one_core"] = {"value": v1, "cores": 1, "sample": f"first {s1} steps ({t1:.1f} s)"}
    vb, sb, tb = _oracle_rate(D, u0, extra_seconds, theta=6.4, stop_tol=1e-13)
    variants["gpu_matched_tolerance"] = {"value": vb, "cores": cores,
                                         "sample": f"first {sb} steps ({tb:.1f} s), theta 6.4, tail bound 1e-13"}
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {steps} of the {NSTEPS} steps of the {D.shape[0]}^3 run "
                      f"({dt:.1f} s, FP64 oracle, theta 0.5, tail bound 1e-18)",
            "variants": variants}


def run_config(args, world, precision):
    """The workload as both arms state it (the same keys and values)."""
    return {"workload": WORKLOAD, "grid": [args.grid] * 3, "steps_per_run": args.nsteps, "tau_days": TAU,
            "operator": "conservative", "scheme": "rosenbrock", "precision": precision,
            "l2": "GPU arm: 256 MiB buffer written between bench steps (inside the timed region); "
                  "CPU arm: not applicable",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2402_02273_gb300 import phantom
    D, u0 = phantom.case(args.grid, seed=0, noise=NOISE)
    P = oracle.Problem(D, rho=RHO)
    u = u0.copy()
    for _ in range(args.warmup):
        u, _ = P.run(u, TAU, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u, _ = P.run(u, TAU, 1)
    dt = time.perf_counter() - t0
    n = D.size
    value = n * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": run_config(args, world, "f64"),
        "sample": "one time step of the 100-step run per bench step",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                         "sample": f"time steps {args.warmup + 1}..{args.warmup + args.steps} of the "
                                   f"{args.grid}^3 run, one per bench step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


L2_BYTES = 129e6  # GB300 L2
# bytes of one value of each form; a term chain works on three weight fields,
# the diagonal, b and two term vectors (Horner sub-step), plus two running-sum
# vectors when there are later sub-steps
VALUE_BYTES = {"f64": 8, "df64": 8, "f32": 4}
# a chain counts as L2-resident when its fields fit in half the L2: the L2 is
# two partitions, one per die, and lines read from both dies are held in both
L2_RESIDENT_BYTES = L2_BYTES / 2


def l2_peak_gbs(et, stream):
    """Best streaming bandwidth (read + write bytes per second) of the
    library's probe with every buffer in the L2 (working sets of 24 to 56 MB,
    under half the L2): a copy, and six inputs to one output, the read/write
    mix of a stencil term.  The denominator for kernels whose working set is
    L2-resident, beside the HBM copy peak."""
    copy = max(et.probe_stream(mb << 20, 1, reps=100, stream=stream) for mb in (12, 16, 24, 28))
    mix = max(et.probe_stream(mb << 20, 6, reps=100, stream=stream) for mb in (4, 6, 8))
    return max(copy, mix), {"copy": copy, "six_in_one_out": mix}


def measure_form(et, torch, D, u0, precision, args, stream, flush, timing=True, every_row=False):
    """Times K bench steps of one precision form; returns a dict of numbers."""
    n = D.size
    g = et.Grid(D.shape, precision=precision, stream=stream)
    Dd = torch.from_numpy(D).to("cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.set_coeffs(Dd, rho=RHO, single_terms=args.single_terms, every_row=every_row or args.every_row)
    setup_ms = (time.perf_counter() - t0) * 1e3
    u0d = torch.from_numpy(u0).to("cuda")
    u = torch.empty_like(u0d)
    s, m, mu, theta = g.schedule(TAU)
    g.enable_timing(timing)

    def one_step():
        u.copy_(u0d)
        g.run(u, TAU, args.nsteps)
        flush.add_(1)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step()
        g.sync_info()
        torch.cuda.synchronize()
        return g, one_step, {"setup_ms": setup_ms, "s": s, "m": m, "mu": mu, "theta": theta}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    rank, world, local = dist_env()
    import torch
    import paper_2402_02273_gb300 as et
    from paper_2402_02273_gb300 import phantom

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev_index = torch.cuda.current_device()
    et.load()
    D, u0 = phantom.case(args.grid, seed=rank, noise=NOISE)
    n = D.size

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(D, u0)

    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    fp64_peak, fp32_peak = et.probe_alu(stream)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    l2_peak, l2_probes = l2_peak_gbs(et, stream)
    hbm_probe = et.probe_stream(1 << 30, 1, reps=5, stream=stream)  # this run's own HBM copy, for context

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(step_fn):
        barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(dev_index) if rank == 0 else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(args.steps):
                step_fn()
            e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        ms = max_over_ranks(e0.elapsed_time(e1) / args.steps)
        barrier()
        return ms, clocks

    def time_form(Dg, ug, prec, every_row=False):
        """K timed runs of one precision form on grid Dg from ug; a result dict."""
        ng = Dg.size
        edge = Dg.shape[0]
        every_row = every_row or args.every_row
        g, step_fn, info = measure_form(et, torch, Dg, ug, prec, args, stream, flush, every_row=every_row)
        ms, clocks = timed(step_fn)
        term_ms, term_launches, other_launches = g.timing()  # last run of the timed region
        rec = g.sync_info()
        avg_launch_ms = term_ms / max(term_launches, 1)
        s_, m_ = info["s"], info["m"]
        kname, pairs = term_kernel_of(prec, args.single_terms, ng)
        # the one-term kernels skip the stencil in rows without off-diagonal entries
        zk = ZERO_ROW_KERNELS.get(kname)
        zero_frac = g.zero_row_voxels() / ng if (zk is not None and not every_row) else 0.0
        nl, vb, vf = launch_mix(prec, s_, m_, pairs, zero_frac, zero_flops=bool(zk))
        bytes_per_launch = vb / nl * ng
        flops_per_launch = vf / nl * ng
        achieved_gbs = bytes_per_launch / (avg_launch_ms * 1e-3) / 1e9
        achieved_tflops = flops_per_launch / (avg_launch_ms * 1e-3) / 1e12
        value = whole_job_rate(world, ng, args.nsteps, ms)
        alu_peak = fp64_peak if prec == "f64" else fp32_peak
        traffic = term_traffic(prec, kname, edge, ng)
        alu_frac = achieved_tflops / alu_peak
        hbm_frac = achieved_gbs / hbm_peak
        # the fields of the term chain (the weights, diagonal, b and the
        # vectors) against the L2: where they fit, the chain runs from the L2
        # and its bandwidth is set against the L2 copy peak of this run
        chain_bytes = VALUE_BYTES[prec] * (7 if s_ == 1 else 9) * ng
        l2_resident = chain_bytes < L2_RESIDENT_BYTES
        if prec == "f64" and alu_frac >= hbm_frac:
            roof = {"bound": "alu", "achieved": achieved_tflops, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": alu_frac, "traffic": traffic,
                    "peak_source": "measured FP64 FMA rate (et_probe_alu, this run)"}
        elif l2_resident:
            roof = {"bound": "l2", "achieved": achieved_gbs, "peak": l2_peak, "unit": "GB/s",
                    "frac": achieved_gbs / l2_peak, "traffic": traffic,
                    "peak_source": "measured L2-resident streaming probe (et_probe_stream, this run)"}
        else:
            roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": hbm_frac, "traffic": traffic, "peak_source": f"{hbm_src} (MEASURED_PEAKS.json)"}
        roof.update({"kernel": kname + (" (two terms per launch)" if pairs else ""),
                     "avg_launch_us": avg_launch_ms * 1e3, "launches_per_run": term_launches,
                     "algorithmic_bytes_per_launch": bytes_per_launch,
                     "algorithmic_flops_per_launch": flops_per_launch, "chain_field_bytes": chain_bytes,
                     "zero_row_fraction": zero_frac, "every_row": every_row,
                     "l2_resident": l2_resident, "l2_peak_gbs": l2_peak, "l2_frac": achieved_gbs / l2_peak,
                     "hbm_frac": hbm_frac, "hbm_achieved_gbs": achieved_gbs, "alu_frac": alu_frac})
        # the launch's time at each peak on its own and the larger of the two:
        # the kernel cannot beat either, so max / measured is its fraction of
        # the combined bound (zero rows are memory work, the others FP64 work)
        t_alu_us = flops_per_launch / (alu_peak * 1e12) * 1e6
        t_mem_us = bytes_per_launch / ((l2_peak if roof["bound"] == "l2" else hbm_peak) * 1e9) * 1e6
        roof["bound_us"] = {"alu": t_alu_us, "memory": t_mem_us}
        roof["combined_frac"] = max(t_alu_us, t_mem_us) / (avg_launch_ms * 1e3)
        # stencil applications per time step: the residual and s m - 1 Taylor terms
        matvecs = s_ * m_
        roof["matvecs_per_step"] = matvecs
        roof["gvoxel_matvecs_per_s"] = ng * matvecs * args.nsteps / (ms * 1e-3) / 1e9
        g.enable_timing(False)
        del g
        torch.cuda.empty_cache()
        return {"value": value, "ms_per_step": ms, "clocks": clocks, "roofline": roof,
                "launches_per_run": term_launches + other_launches, "info": info,
                "final_mass": rec["mass"], "final_umax": rec["umax"], "grid": [edge] * 3}

    results = {}
    forms = ["f64"] if args.no_forms else [f for f in args.forms.split(",") if f]
    for prec in forms:
        results[prec] = time_form(D, u0, prec)

    # the same forms with the stencil evaluated in every row (no zero-row
    # skip): the work of a dense 7-point operator, for comparison
    every = {}
    if not args.no_forms and not args.every_row:
        for prec in [f for f in args.every_row_forms.split(",") if f]:
            every[prec] = time_form(D, u0, prec, every_row=True)

    # the FP32 and DF64 forms on a grid whose chain is far beyond the L2, where
    # the HBM fraction applies (the same phantom type and run, larger grid)
    large = {}
    if args.large_grid and not args.no_forms:
        Dl, ul = phantom.case(args.large_grid, seed=rank, noise=NOISE)
        for prec in [f for f in args.large_forms.split(",") if f]:
            large[prec] = time_form(Dl, ul, prec)
        del Dl, ul

    # adjoint form: one gradient = forward run of ADJ_STEPS steps keeping
    # checkpoints every ADJ_CK steps + the reverse pass from them (the misfit
    # cotangent u_K - u_target is the caller's, one torch subtraction)
    adjoint = {}
    if not args.no_adjoint and not args.no_forms:
        for prec in [f for f in args.adjoint_forms.split(",") if f]:
            g = et.Grid(D.shape, precision=prec, stream=stream)
            g.set_coeffs(torch.from_numpy(D).to("cuda"), rho=RHO)
            u0d = torch.from_numpy(u0).to("cuda")
            tgt = u0d * 0.5
            u = torch.empty_like(u0d)

            ws = g.adjoint_workspace(TAU, ADJ_STEPS, ADJ_CK)

            def adj_step():
                # one gradient: the forward run keeps the checkpoints, the
                # reverse pass starts from them
                u.copy_(u0d)
                g.run_checkpointed(u, TAU, ADJ_STEPS, ADJ_CK, workspace=ws)
                g.vjp_checkpointed(ws, TAU, ADJ_STEPS, u - tgt, ADJ_CK)
                flush.add_(1)

            with torch.cuda.stream(stream):
                for _ in range(args.warmup):
                    adj_step()
            ms, clocks = timed(adj_step)
            adjoint[prec] = {"value": whole_job_rate(world, n, ADJ_STEPS, ms), "unit": UNIT,
                             "ms_per_gradient": ms, "steps": ADJ_STEPS, "checkpoint_every": ADJ_CK,
                             "note": "voxel-steps of the forward run per second of forward + adjoint",
                             "clocks": clocks}
            del g
            torch.cuda.empty_cache()

    # batched form: BATCH_COUNT uneven grids (phantom.batch_case, seeds 1000 + i,
    # offset per rank) in one CUDA graph of batched launches, 100 steps; one
    # warm-up run (autotune + graph capture), then --batch-runs timed runs
    batch = {}
    if not args.no_batch and not args.no_forms:
        cases = [phantom.batch_case(i, base_seed=1000 + rank * args.batch_count) for i in range(args.batch_count)]
        shapes = [c["D"].shape for c in cases]
        rhos = [c["rho"] for c in cases]
        Dcat = torch.from_numpy(np.concatenate([c["D"].ravel() for c in cases])).to("cuda")
        ucat0 = torch.from_numpy(np.concatenate([c["u0"].ravel() for c in cases])).to("cuda")
        nb = int(Dcat.numel())
        del cases
        for prec in [f for f in args.batch_forms.split(",") if f]:
            B = et.Batch(shapes, precision=prec, stream=stream)
            t0 = time.perf_counter()
            B.set_coeffs(Dcat, rhos, every_row=args.every_row)
            setup_ms = (time.perf_counter() - t0) * 1e3
            variant, tune_us = B.autotune(TAU)
            s_list, m_list = B.schedule(TAU)
            u = torch.empty_like(ucat0)

            def batch_step():
                u.copy_(ucat0)
                B.run(u, TAU, args.nsteps)

            with torch.cuda.stream(stream):
                batch_step()
            B.sync_info()
            torch.cuda.synchronize()
            ksave = args.steps
            args.steps = args.batch_runs
            ms, clocks = timed(batch_step)
            args.steps = ksave
            recs = B.sync_info()
            sizes = [int(np.prod(sh)) for sh in shapes]
            # the autotuned variant: two terms per launch in the first half of
            # the index range (F32 / DF64)
            pairs = prec != "f64" and variant < len(tune_us) // 2
            if not pairs:
                bkernel = "batch_term_f64_kernel" if (prec == "f64" and variant == 0) else \
                    ("batch_term_df64_kernel" if prec == "df64" else "batch_term_kernel")
            else:
                bkernel = "batch_term2_quad_kernel" if prec == "f32" else "batch_term2_kernel"
            # voxels in rows without off-diagonal entries, per grid, where the
            # chosen kernel skips them
            zk = ZERO_ROW_KERNELS.get(bkernel)
            zrows = B.zero_row_voxels() if zk is not None else [0] * len(sizes)
            zfr = [z_i / n_i for z_i, n_i in zip(zrows, sizes)]
            zf_all = sum(zrows) / nb
            # algorithmic bytes of the term launches over the whole run, per grid
            term_bytes = sum(n_i * launch_mix(prec, s_i, m_i, pairs, z_i, bool(zk))[1]
                             for n_i, s_i, m_i, z_i in zip(sizes, s_list, m_list, zfr)) * args.nsteps
            gbs = term_bytes / (ms * 1e-3) / 1e9
            # the autotuner's timing of the chosen variant on the first launch
            # of every grid (Horner terms), per term; cold L2 is not enforced
            # between its repeats: the launch streams 4-8 GB, far above L2
            t_us = tune_us[variant]
            # one Horner term (pair: one launch) over all grids, zero rows at their cost
            _, hb_v, hf_v = launch_mix(prec, 1, 3 if pairs else 2, pairs, zf_all, bool(zk))
            if prec == "f64":
                ach = hf_v * nb / (t_us * 1e-6) / 1e12
                hbm_b = hb_v * nb / (t_us * 1e-6) / 1e9
                broof = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": ach / fp64_peak, "hbm_frac": hbm_b / hbm_peak}
            else:
                per_term = hb_v / (2.0 if pairs else 1.0)
                ach = per_term * nb / (t_us * 1e-6) / 1e9
                broof = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak}
            broof.update({"zero_row_fraction": zf_all, "kernel": bkernel + (" (two terms per launch" if pairs else " (one term per launch")
                          + ", first launch of every grid)", "us_per_term": t_us,
                          "traffic": term_traffic(prec, bkernel, "batch", nb),
                          "algorithmic_bytes_per_launch": hb_v * nb,
                          "launch_us": t_us * (2.0 if pairs else 1.0)})
            batch[prec] = {"value": whole_job_rate(world, nb, args.nsteps, ms), "unit": UNIT,
                           "ms_per_run": ms, "voxels": nb, "grids": len(shapes), "steps": args.nsteps,
                           "setup_ms": setup_ms, "variant": variant, "two_terms_per_launch": pairs,
                           "autotune_us_per_term": tune_us,
                           "s_range": [min(s_list), max(s_list)], "m_range": [min(m_list), max(m_list)],
                           "roofline": broof, "term_gbs_whole_run": gbs, "term_hbm_frac_whole_run": gbs / hbm_peak,
                           # stencil applications (residual + s m - 1 terms) per step over all grids,
                           # and their rate over the whole run: the batch's own schedules differ
                           # from the single grid's (m from its rho and D scale)
                           "matvecs_per_voxel_step": sum(n_i * s_i * m_i for n_i, s_i, m_i
                                                         in zip(sizes, s_list, m_list)) / nb,
                           "gvoxel_matvecs_per_s": sum(n_i * s_i * m_i for n_i, s_i, m_i
                                                       in zip(sizes, s_list, m_list)) * args.nsteps
                                                   / (ms * 1e-3) / 1e9,
                           # per step: residual, the longest chain's launches, stats
                           "launches_per_run": args.nsteps * (max(launch_mix(prec, si, mi, pairs)[0]
                                                                  for si, mi in zip(s_list, m_list)) + 2),
                           "max_final_umax": max(r["umax"] for r in recs),
                           "timed_runs": args.batch_runs, "warmup_runs": 1, "clocks": clocks}
            B.close()
            del B, u
            torch.cuda.empty_cache()
        del Dcat, ucat0
        torch.cuda.empty_cache()

    # Crank-Nicolson comparison (Sec. 2.3 / Table 2 of the paper): the same
    # 128^3 run of 100 steps by Crank-Nicolson steps (FP64 conjugate gradients
    # to a relative residual of --cn-rtol), and the time-discretisation error
    # of both schemes at the end of the run against the exponential step at
    # tau / 16 (untimed)
    crank = None
    if not args.no_cn and not args.no_forms:
        g = et.Grid(D.shape, precision="f64", stream=stream)
        g.set_coeffs(torch.from_numpy(D).to("cuda"), rho=RHO)
        u0d = torch.from_numpy(u0).to("cuda")
        u = torch.empty_like(u0d)
        info = g.info_buffer(args.nsteps)

        def cn_step():
            u.copy_(u0d)
            g.cn_run(u, TAU, args.nsteps, rtol=args.cn_rtol, info=info)
            flush.add_(1)

        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                cn_step()
        g.sync_info()
        ms, clocks = timed(cn_step)
        g.sync_info()
        iters = g.decode_info(info)["m"]
        u_cn = u.cpu().numpy()
        # the exponential step's run and the fine reference, untimed
        with torch.cuda.stream(stream):
            v = u0d.clone()
            g.run(v, TAU, args.nsteps)
            ref = u0d.clone()
            g.run(ref, TAU / 16, 16 * args.nsteps)
        g.sync_info()
        u_exp, u_ref = v.cpu().numpy(), ref.cpu().numpy()
        scale = np.abs(u_ref).max()
        value = whole_job_rate(world, n, args.nsteps, ms)
        crank = {"value": value, "unit": UNIT, "ms_per_run": ms, "rtol": args.cn_rtol,
                 "cg_iterations_per_step": [int(iters.min()), int(iters.max())],
                 "cg_iteration_cap": g.cn_iteration_cap(TAU, args.cn_rtol),
                 # stencil applications per step: the residual and one per iteration
                 "gvoxel_matvecs_per_s": n * (float(iters.mean()) + 1) * args.nsteps / (ms * 1e-3) / 1e9,
                 "exponential_value": results["f64"]["value"] if "f64" in results else None,
                 "max_error_vs_tau16_reference": {"crank_nicolson": float(np.abs(u_cn - u_ref).max() / scale),
                                                  "exponential": float(np.abs(u_exp - u_ref).max() / scale)},
                 "clocks": clocks,
                 "note": "FP64 both; errors at t = 730 d relative to max|u|, reference = exponential step, tau/16"}
        del g
        torch.cuda.empty_cache()

    # end to end through the public API with host buffers (pinned): H2D of D and
    # u0, coefficient setup, the 100-step run, D2H of u and of the last record
    e2e = None
    if True:
        g = et.Grid(D.shape, precision="f64", stream=stream)
        D_pin = torch.from_numpy(D).pin_memory().numpy()
        u_pin = torch.empty(n, dtype=torch.float64).pin_memory().numpy()

        def e2e_step():
            u_pin[:] = u0.ravel()
            g.set_coeffs(D_pin, rho=RHO)
            g.run_host(u_pin, TAU, args.nsteps)

        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                e2e_step()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps)
        e2e = {"value": whole_job_rate(world, n, args.nsteps, e2e_ms), "unit": UNIT,
               "h2d_bytes_per_step": 2 * 8 * n, "d2h_bytes_per_step": 8 * n + 40,
               "ms_per_step": e2e_ms,
               "path": "et_set_coeffs_host + et_run_host (pinned host buffers, host wall clock)"}
        del g

    if rank == 0:
        head = forms[0]
        r = results[head]
        line = {
            "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": head, "data": "synthetic",
            "config": run_config(args, world, head),
            "schedule": {"s": r["info"]["s"], "m": r["info"]["m"], "theta": r["info"]["theta"],
                         "tol": 1e-7 if head == "f32" else 1e-13, "setup_ms": r["info"]["setup_ms"]},
            "roofline": r["roofline"],
            "clocks": r["clocks"],
            "gpu_launches": args.steps * r["launches_per_run"],
            "e2e": e2e,
            "cpu_baseline": base,
            "alu_peaks_tflops": {"fp64": fp64_peak, "fp32": fp32_peak},
            "adjoint": adjoint,
            "batch": batch,
            "forms": {p: {"value": results[p]["value"], "ms_per_step": results[p]["ms_per_step"],
                          "dtype": p, "s": results[p]["info"]["s"], "m": results[p]["info"]["m"],
                          "roofline": results[p]["roofline"], "clocks": results[p]["clocks"]}
                      for p in results},
            "forms_large_grid": {p: {"value": large[p]["value"], "ms_per_step": large[p]["ms_per_step"],
                                     "grid": large[p]["grid"], "dtype": p, "s": large[p]["info"]["s"],
                                     "m": large[p]["info"]["m"], "roofline": large[p]["roofline"],
                                     "clocks": large[p]["clocks"]}
                                 for p in large},
            "forms_every_row": {p: {"value": every[p]["value"], "ms_per_step": every[p]["ms_per_step"],
                                    "dtype": p, "roofline": every[p]["roofline"], "clocks": every[p]["clocks"]}
                                for p in every},
            "stream_probe_gbs": {"l2": l2_peak, "l2_probes": l2_probes, "hbm_copy_1gib": hbm_probe},
            "crank_nicolson": crank,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
