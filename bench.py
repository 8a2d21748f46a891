#!/usr/bin/env python
"""Benchmark: RAS-Jacobi smoothing throughput on one GB300 (or N replicas).

Workload (one "step"): the 8192 x 8192 layered sinker (10 seeded horizontal
layers with log10 eta ~ U[-3, 3] plus a centred sinker, viscosity contrast up
to 1e6, unit square, free-slip walls), FP32: 100 RAS-Jacobi sweeps (48 x 64
tiles, k = 8 local sweeps, overlap k-1 = 7, SplitMix64 tile shifts; with
overlap k-1 the map is exactly global Jacobi whatever the tile, and 48 x 64
with k = 8 is the fastest exact schedule measured), then the energy residual
norm (FP64 accumulation, three scalars back to the host).  One cell-update =
vx and vy of one cell updated once; value = nx * ny * sweeps * steps / time.

Every field is 268 MB (FP32), so the 8 fields of a sweep (2.1 GB) are far
larger than the 129 MB L2: inputs larger than L2, no flush needed.

--impl reference times the FP64 CPU oracle on this host's cores on a bounded
sample of the same workload (see cpu_sample below).
"""
import argparse
import hashlib
import json
import math
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RAS-Jacobi Gcell-updates/s + % HBM peak; time to 1e-8 residual FP32 vs FP64"
UNIT = "Gcell-updates/s"
WORDS_PER_CELL_SWEEP = 8  # read vx, vy, eta_c, eta_n, bx, by; write vx, vy
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0
# FP32 tile-kernel arithmetic per cell-sweep (an FMA counts 2): fluxes
# sigma'xx, sigma'yy (2 + 2), the node shear (6) scaled twice (2), M v in x
# and y (3 + 3), the two damped updates (3 + 3); the general form's count,
# kept as the algorithmic figure on square cells too, where the kernel forms
# the scaled shear in 4
FLOPS_PER_CELL_SWEEP = 24
# nominal arithmetic peaks of the GB300 (152 SMs at 2.07 GHz): FP32 128 lanes
# per SM, an FMA counting 2 flops; FP64 at its nominal 1.25 TFLOP/s
NOMINAL_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
NOMINAL_FP64_TFLOPS = 1.25
RAS_SOURCES = ["paper_2509_19061_gb300/csrc/ras_kernels.cu", "paper_2509_19061_gb300/csrc/stencil.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--sweeps", type=int, default=100)
    ap.add_argument("--tile", type=int, nargs=2, default=[48, 64])
    ap.add_argument("--k", type=int, default=8)
    ap.add_argument("--overlap", type=int, default=None)
    ap.add_argument("--no-extras", action="store_true", help="skip the variant table, e2e and CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--solve-n", type=int, default=4096, help="grid of the time-to-1e-8 solve")
    ap.add_argument("--batch", type=int, default=256, help="instances of the batched workload (0: skip)")
    ap.add_argument("--c2-sweeps", type=int, default=100, help="sweeps per smoother in the 1024^2 FP64 table")
    ap.add_argument("--uzawa-n", type=int, default=1024, help="grid of the Uzawa Stokes solve")
    ap.add_argument("--robust-n", type=int, default=256, help="grid of the smoother robustness comparison")
    ap.add_argument("--n3d", type=int, default=384, help="cells per side of the 3D smoothing leg")
    ap.add_argument("--only", choices=["solve", "batch", "autotune", "c2", "uzawa", "robustness", "fp32err",
                                       "smoothers", "smooth3d", "slabs"],
                    help="run one extra leg alone and print its JSON (for profiling it)")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def source_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_entry(key, src_hash):
    """The committed ncu summary entry of this launch shape, if it was taken
    on the current kernel source; None otherwise."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[key]
        return e if e.get("source_hash") == src_hash else None
    except Exception:
        return None


def ncu_traffic(key, src_hash):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; None otherwise."""
    e = ncu_entry(key, src_hash)
    try:
        return None if e is None else float(e["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        exe = shutil.which("nvidia-smi")
        if exe:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen([exe, "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def host_cpu():
    """CPU model and core count of this host (lscpu / nproc equivalents)."""
    model = "unknown"
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"model": model, "nproc": os.cpu_count()}


def cpu_sample(args, target_s):
    """Time the FP64 oracle's RAS-Jacobi on the same workload generator at
    1024^2 (same tiles, k, overlap, shifts) for about target_s seconds."""
    import oracle as ora
    from paper_2509_19061_gb300 import inputs
    n = 1024
    prob = inputs.layered_sinker(n, seed=4)
    g = ora.Grid(n, n, prob.hx, prob.hy, prob.eta_c, prob.eta_n)
    bx, by = ora.rhs(g, prob.fx, prob.fy, None)
    k = args.k
    o = args.overlap if args.overlap is not None else k - 1
    t0 = time.perf_counter()
    ora.ras(g, bx, by, 0.3, k, args.tile[0], args.tile[1], k, o, shift_mode=1, seed=1)
    t_one = max(time.perf_counter() - t0, 1e-3)
    outer = max(1, int(target_s / t_one))
    sweeps = outer * k
    t0 = time.perf_counter()
    ora.ras(g, bx, by, 0.3, sweeps, args.tile[0], args.tile[1], k, o, shift_mode=1, seed=1)
    dt = time.perf_counter() - t0
    return {"value": n * n * sweeps / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "host": host_cpu(),
            "sample": "FP64 C oracle, single thread, layered sinker %dx%d (same generator, seed 4), RAS %dx%d "
                      "tiles k=%d overlap=%d, %d sweeps in %.1f s" % (n, n, args.tile[0], args.tile[1], k, o,
                                                                      sweeps, dt),
            "seconds": dt}


def cpu_sample_all_cores(args, target_s, reps=5):
    """The OpenMP build of the same oracle source (the tiles of an outer
    iteration in parallel) on every host core: the same RAS sample as
    cpu_sample, `reps` repetitions of about target_s / reps seconds each;
    median and the range of the repetitions."""
    import oracle as ora
    from paper_2509_19061_gb300 import inputs
    n = 1024
    prob = inputs.layered_sinker(n, seed=4)
    g = ora.Grid(n, n, prob.hx, prob.hy, prob.eta_c, prob.eta_n)
    bx, by = ora.rhs(g, prob.fx, prob.fy, None)
    k = args.k
    o = args.overlap if args.overlap is not None else k - 1
    t0 = time.perf_counter()
    ora.ras_all_cores(g, bx, by, 0.3, k, args.tile[0], args.tile[1], k, o, shift_mode=1, seed=1)
    t_one = max(time.perf_counter() - t0, 1e-3)
    sweeps = max(1, int(target_s / reps / t_one)) * k
    vals = []
    for _ in range(reps):
        t0 = time.perf_counter()
        ora.ras_all_cores(g, bx, by, 0.3, sweeps, args.tile[0], args.tile[1], k, o, shift_mode=1, seed=1)
        vals.append(n * n * sweeps / (time.perf_counter() - t0) / 1e9)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": statistics.median(vals), "unit": UNIT, "cores": cores, "kind": "oracle (OpenMP build)",
            "range": [min(vals), max(vals)], "reps": reps,
            "sample": "FP64 C oracle built with OpenMP, %d threads, layered sinker %dx%d, RAS %dx%d tiles k=%d "
                      "overlap=%d, %d sweeps per repetition" % (cores, n, n, args.tile[0], args.tile[1], k, o,
                                                                sweeps)}


def cpu_vcycle_solve(api, n=512):
    """The V-cycle solve of the time-to-1e-8 workload on the host, bounded: the
    FP64 oracle's flexible CG around its V-cycle (RAS 32 x 32, k = 4,
    overlap 3, 5/5 sweeps x2.5 per level capped at 40, dense coarsest) to
    E_v <= 1e-8 on the multi-sinker at n^2, one thread; beside it the GPU's
    solve of the same instance with FP64 and with FP32 sweeps (the same
    schedule, FP64 outer flexible CG)."""
    import torch
    import oracle as ora
    from paper_2509_19061_gb300 import inputs
    prob = inputs.multi_sinker(n, seed=3)
    g = ora.Grid(n, n, prob.hx, prob.hy, prob.eta_c, prob.eta_n)
    mg = ora.MG(variant=4, ti=32, tj=32, k=4, overlap=3, nu_max=40, seed=1)
    t0 = time.perf_counter()
    _, _, its, fe, _ = ora.mg_fcg(g, prob.fx, prob.fy, None, mg, 1e-8, 200)
    cpu_s = time.perf_counter() - t0
    out = {"workload": "multi_sinker_%dx%d_seed3" % (n, n), "tol": 1e-8,
           "oracle": {"seconds": cpu_s, "cycles": its, "final_energy_residual": fe, "cores": 1}}
    ctx = api.StokesContext(n, n, 1.0, 1.0, "f64")
    ctx.set_problem(prob)
    vx, vy = ctx.field(), ctx.field()
    for inner in ("f64", "f32"):
        kw = dict(variant="ras", tile=(32, 32), k=4, overlap=3, seed=1, nu_max=40, inner=inner, krylov=True,
                  tol=1e-8, max_cycles=200)
        ctx.vcycle(vx, vy, None, **kw)
        vx.zero_()
        vy.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, e, cyc = ctx.vcycle(vx, vy, None, **kw)
        torch.cuda.synchronize()
        out["gpu_" + inner + "_inner"] = {"seconds": time.perf_counter() - t0, "cycles": cyc, "final_energy_residual": e,
                                          "status": st}
    ctx.close()
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_sample(args, per_step / 4)
    vals, secs = [], []
    for _ in range(args.steps):
        r = cpu_sample(args, per_step)
        vals.append(r["value"])
        secs.append(r["seconds"])
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.median(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": r["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def workload_config(args):
    o = args.overlap if args.overlap is not None else args.k - 1
    return {"workload": "layered_sinker_%dx%d_contrast1e6_ras_%s" % (args.n, args.n, args.dtype),
            "nx": args.n, "ny": args.n, "tile": list(args.tile), "k": args.k, "overlap": o,
            "sweeps_per_step": args.sweeps, "shifts": "splitmix64", "omega": 0.3,
            "l2": "inputs larger than L2 (8 fields x %.0f MB per sweep), no flush" % (
                (args.n + 1) * (args.n + 1) * (4 if args.dtype == "f32" else 8) / 1e6),
            "step": "b = f - G p, %d RAS sweeps, energy norm" % args.sweeps}


TILE_KERNEL_NAMES = {"pair": "k_ras_pair", "tma": "k_ras_tma", "global": "k_ras_reg", "shared": "k_ras"}


def tile_kernel_name(api, n, tile, overlap, dt_name):
    """Name of the tile kernel the library picks for this launch shape."""
    return TILE_KERNEL_NAMES[api.stokes_tile_kernel_plan(n, n, tuple(tile), overlap, dt_name)[0]]


def median_ci(xs):
    """Median of the per-step times with its distribution-free 95% confidence
    interval (order statistics n/2 -+ 0.98 sqrt(n), 1-based)."""
    v = sorted(xs)
    n = len(v)
    if n == 0:
        return None
    lo = max(int(math.floor(n / 2 - 0.98 * math.sqrt(n))), 1)
    hi = min(int(math.ceil(n / 2 + 1 + 0.98 * math.sqrt(n))), n)
    return {"median": statistics.median(v), "ci95": [v[lo - 1], v[hi - 1]], "n": n, "unit": "ms"}


def max_over_ranks(x, world, device):
    """The largest x over all ranks, returned on every rank (x itself when
    world == 1).  NCCL on the GPU machine; the CPU tests use gloo."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, cells, sweeps, steps, ms_total):
    """Whole-job Gcell-updates/s: every rank smooths its own replica of the
    workload, so the job processes world x cells x sweeps x steps updates in
    the slowest rank's time."""
    return world * cells * sweeps * steps / (ms_total / 1e3) / 1e9


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2509_19061_gb300 import api, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    # all work on a created stream: kernels on the legacy default stream would
    # wait for the copies the end-to-end leg runs on its own streams
    torch.cuda.set_stream(torch.cuda.Stream())
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    n, dt_name = args.n, args.dtype
    k = args.k
    o = args.overlap if args.overlap is not None else k - 1
    prob = inputs.layered_sinker(n, seed=4)
    stream = torch.cuda.current_stream()
    ctx = api.StokesContext(n, n, 1.0, 1.0, dt_name, stream=stream)
    ctx.set_problem(prob)
    vx, vy = ctx.field(), ctx.field()
    cells = n * n
    esize = 4 if dt_name == "f32" else 8

    def step(s, seed):
        ctx.smooth(vx, vy, None, variant="ras", sweeps=s, tile=tuple(args.tile), k=k, overlap=o, seed=seed)
        return ctx.energy(vx, vy)

    for w in range(args.warmup):
        step(args.sweeps, 1000 + w)
    torch.cuda.synchronize()
    ctx.profile_reset(timing=True)
    barrier()
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    e0, e1 = evs[0], evs[-1]
    with ClockSampler(local) as clk:
        e0.record(stream)
        for it in range(args.steps):
            energy = step(args.sweeps, it)
            evs[it + 1].record(stream)
        torch.cuda.synchronize()
    barrier()
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    ms_total = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    prof = ctx.profile()
    launches = sum(v[0] for v in prof.values())
    ras_launches, ras_groups, ras_ms = prof["ras"]
    ms_step = ms_total / args.steps
    value = job_value(world, cells, args.sweeps, args.steps, ms_total)

    # roofline of the dominant kernel (the RAS tile kernel).  One launch runs
    # sweeps_per_launch local sweeps over every cell (the last launch of a step
    # runs the remainder).  Its bound is the FP32 (FP64) pipe, not HBM (ncu:
    # issue- and FMA-pipe-bound, DRAM well below peak), so the roofline is the
    # arithmetic one: algorithmic flops of the owned cells per launch over the
    # nominal arithmetic peak.  The HBM view is reported beside it twice: the
    # launch's minimum DRAM bytes (each field read once, vx and vy written
    # once: 8 words per cell per launch), and the effective bytes of the
    # paper's yardstick (8 words per cell per sweep, which exceeds the HBM
    # peak when k > 1 because the window stays on chip for k sweeps).
    sweeps_per_launch = args.sweeps / math.ceil(args.sweeps / k)
    min_bytes = WORDS_PER_CELL_SWEEP * esize * cells
    eff_bytes = min_bytes * sweeps_per_launch
    avg_ms = ras_ms / max(ras_groups, 1)
    avg_s = avg_ms / 1e3
    peak, peak_kind = measured_peaks()
    key = "ras_%s_%d_t%dx%d_k%d_o%d" % (dt_name, n, args.tile[0], args.tile[1], k, o)
    traffic = ncu_traffic(key, source_hash(RAS_SOURCES))
    limiter = (ncu_entry(key, source_hash(RAS_SOURCES)) or {}).get("limiter")
    flops = FLOPS_PER_CELL_SWEEP * cells * sweeps_per_launch
    tflops = flops / avg_s / 1e12
    alu_peak = NOMINAL_FP32_TFLOPS if dt_name == "f32" else NOMINAL_FP64_TFLOPS
    hbm_min = min_bytes / avg_s / 1e9
    hbm_eff = eff_bytes / avg_s / 1e9
    peak_src = ("%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind) if peak_kind == "measured" else "fallback 6800 GB/s"
    alu_bound = k > 1
    if alu_bound:
        roofline = {"bound": "alu", "achieved": tflops, "peak": alu_peak, "unit": "TFLOP/s", "frac": tflops / alu_peak,
                    "traffic": traffic,
                    "peak_source": "nominal %s: 152 SMs x %s x 2.07 GHz" % (
                        dt_name, "128 FP32 lanes x 2 flops per FMA" if dt_name == "f32" else "FP64 1.25 TFLOP/s"),
                    "algorithmic_flops_per_launch": flops}
    else:
        roofline = {"bound": "hbm", "achieved": hbm_min, "peak": peak, "unit": "GB/s", "frac": hbm_min / peak,
                    "traffic": traffic, "peak_source": peak_src, "algorithmic_bytes_per_launch": min_bytes}
    roofline.update({
        "kernel": tile_kernel_name(api, n, args.tile, o, dt_name), "kernel_avg_ms": avg_ms,
        "kernel_share": ras_ms / ms_total, "sweeps_per_launch": sweeps_per_launch,
        "flops_per_cell_sweep": FLOPS_PER_CELL_SWEEP, "limiter": limiter,
        "traffic_note": "traffic = dram__bytes_read.sum + dram__bytes_write.sum per launch from the committed "
                        "ncu summary, null unless taken on the current kernel source",
        "hbm_min": {"achieved": hbm_min, "peak": peak, "unit": "GB/s", "frac": hbm_min / peak,
                    "bytes_per_launch": min_bytes, "peak_source": peak_src,
                    "note": "the launch's minimum DRAM traffic: 8 words per cell per launch (6 fields read "
                            "once, vx and vy written once)"},
        "effective": {"achieved": hbm_eff, "peak": peak, "unit": "GB/s", "frac": hbm_eff / peak,
                      "frac_nominal": hbm_eff / NOMINAL_HBM_GBS, "bytes_per_launch": eff_bytes,
                      "note": "the paper's yardstick, 8 words per cell per sweep; exceeds 1 with k > 1 "
                              "(temporal blocking), so it is not a roofline fraction"},
        "dram_bytes_per_cell_launch": None if traffic is None else traffic / cells,
    })

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dt_name, "data": "synthetic (seeded layered sinker, no dataset)",
            "config": dict(workload_config(args), parallelism="replicas%d" % world if world > 1 else "single"),
            "gpu_launches": launches, "roofline": roofline, "clocks": clk.summary(),
            "step_ms": median_ci(step_ms),
            "energy_residual_after_step": (energy[0] / energy[2]) ** 0.5}

    if not args.no_extras:
        # every rank runs the end-to-end step (slowest rank's time counts)
        e2e = e2e_measure(args, ctx, prob, stream, world, barrier)
        if rank == 0:
            line["e2e"] = e2e
    # the single-GPU tables (variants, solves, batched workload, tuning, CPU
    # baseline) run at N = 1 only: at N > 1 they would hold every GPU while
    # rank 0 alone works
    if not args.no_extras and world == 1:
        line["fp32_vs_fp64"] = fp32_error_leg(args, api, prob)
        line["variants"] = variant_table(args, api, prob)
        line["c2_f64_1024"] = c2_table(args, api)
        line["time_to_1e-8"] = solve_times(args, api)
        if args.batch > 0:
            line["batched"] = batch_leg(args, api)
        line["autotune"] = autotune_leg(args, api)
        line["uzawa_stokes"] = uzawa_leg(args, api)
        line["smoother_robustness"] = robustness_leg(args, api)
        line["smooth3d"] = smooth3d_leg(args, api)
        line["global_smoothers"] = smoothers_leg(args, api)
        line["slabs"] = slabs_leg(args, api)
        line["cpu_baseline"] = {kk: vv for kk, vv in cpu_sample(args, args.cpu_seconds).items() if kk != "seconds"}
        line["cpu_baseline"]["all_cores"] = cpu_sample_all_cores(args, args.cpu_seconds / 2)
        line["cpu_baseline"]["vcycle_solve"] = cpu_vcycle_solve(api)
    ctx.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def e2e_measure(args, ctx, prob, stream, world, barrier=lambda: None):
    """Same step through the public API with host buffers: every step copies
    all of its inputs (eta_c, eta_n, fx, fy, initial vx, vy) from pinned host
    memory to the device, runs set_viscosity, set_rhs, smooth and the energy
    norm, and copies the smoothed velocity back to pinned host memory, all
    inside the timed region.  Copies run on a separate stream into two
    alternating device buffer sets, so step i+1's inputs travel while step i
    computes (events order each buffer set's reuse)."""
    import torch
    host = {}
    for name, arr in (("eta_c", prob.eta_c), ("eta_n", prob.eta_n), ("fx", prob.fx), ("fy", prob.fy)):
        host[name] = ctx.pack(arr, name).cpu().pin_memory()
    host["vx"] = torch.zeros((ctx.ny + 1, ctx.pitch), dtype=ctx.tdtype).pin_memory()
    host["vy"] = torch.zeros_like(host["vx"]).pin_memory()
    outs = [(torch.empty_like(host["vx"]).pin_memory(), torch.empty_like(host["vx"]).pin_memory())
            for _ in range(2)]
    dev = [{name: ctx.field() for name in host} for _ in range(2)]
    cs = torch.cuda.Stream()  # host -> device
    co = torch.cuda.Stream()  # device -> host (the other direction of the link, concurrently)
    copied = [torch.cuda.Event() for _ in range(2)]
    computed = [torch.cuda.Event() for _ in range(2)]
    drained = [torch.cuda.Event() for _ in range(2)]
    k = args.k
    o = args.overlap if args.overlap is not None else k - 1
    steps = max(2, args.steps)

    def h2d(i):
        # buffer set i % 2 is free once step i - 2's result has left it
        b = dev[i % 2]
        with torch.cuda.stream(cs):
            if i >= 2:
                cs.wait_event(drained[i % 2])
            for name, t in host.items():
                b[name].copy_(t, non_blocking=True)
            copied[i % 2].record(cs)

    def d2h(i):
        b, (ox, oy) = dev[i % 2], outs[i % 2]
        with torch.cuda.stream(co):
            co.wait_event(computed[i % 2])
            ox.copy_(b["vx"], non_blocking=True)
            oy.copy_(b["vy"], non_blocking=True)
            drained[i % 2].record(co)

    def run(n):
        # step i: its kernels are enqueued first, then step i-1's result
        # copy-out and step i+1's inputs copy-in (both overlap step i's
        # kernels; a copy enqueued ahead of a step's kernels held them back
        # until it finished), then step i's energy norm, which synchronises
        h2d(0)
        for i in range(n):
            b = dev[i % 2]
            stream.wait_event(copied[i % 2])
            ctx.set_viscosity_dev(b["eta_c"], b["eta_n"])
            ctx.set_rhs_dev(b["fx"], b["fy"])
            ctx.smooth(b["vx"], b["vy"], None, variant="ras", sweeps=args.sweeps, tile=tuple(args.tile), k=k,
                       overlap=o, seed=i)
            computed[i % 2].record(stream)
            if i >= 1:
                d2h(i - 1)
            if i + 1 < n:
                h2d(i + 1)
            ctx.energy(b["vx"], b["vy"])  # synchronises the context's stream
        d2h(n - 1)
        torch.cuda.synchronize()

    run(2)
    barrier()
    t0 = time.perf_counter()
    run(steps)
    dt = max_over_ranks(time.perf_counter() - t0, world, "cuda")
    h2d_bytes = sum(t.numel() * t.element_size() for t in host.values())
    d2h_bytes = outs[0][0].numel() * outs[0][0].element_size() * 2 + 24
    return {"value": world * args.n * args.n * args.sweeps * steps / dt / 1e9, "unit": UNIT,
            "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": d2h_bytes, "steps": steps,
            "ms_per_step": 1000.0 * dt / steps,
            "pipelining": "step i's kernels enqueued first, then step i-1's result copied out on one stream and "
                          "step i+1's inputs copied in on another while step i computes"}


def solve_times(args, api):
    """Time to a 1e-8 velocity energy residual on the 4096^2 multi-sinker
    (20 seeded inclusions, log10 eta ~ U[-3, 3]): FP64 outer flexible CG
    around a V-cycle (5/5 sweeps x2.5 per level capped at 40, dense FP64
    coarsest) whose sweeps run in FP32 or FP64.  Each precision runs the RAS
    schedule the autotuner picked for its sweeps and the 32 x 32, k = 4,
    overlap 3 schedule (FP32 also exact Jacobi on 48 x 64 tiles, k = 8); its
    time is the fastest of them."""
    import torch
    from paper_2509_19061_gb300 import autotune, inputs
    n = args.solve_n
    prob = inputs.multi_sinker(n, seed=3)
    ctx = api.StokesContext(n, n, 1.0, 1.0, "f64")
    ctx.set_problem(prob)
    out = {"workload": "multi_sinker_%dx%d_seed3" % (n, n), "tol": 1e-8, "outer": "f64 flexible CG",
           "nu": "5/5 x2.5 per level, cap 40"}
    vx, vy = ctx.field(), ctx.field()
    for inner in ("f32", "f64"):
        scheds = [autotune.tuned_smoother(n, n, prob.eta_c, prob.eta_n, inner),
                  dict(variant="ras", tile=(32, 32), k=4, overlap=3)]
        if inner == "f32":
            # exact Jacobi (overlap k - 1) on taller tiles: the same iterates as any
            # other exact-Jacobi schedule, a 64 x 80 window of the pair kernel
            scheds.append(dict(variant="ras", tile=(48, 64), k=8, overlap=7))
        runs = []
        for sm in scheds:
            if any(r["schedule"] == sm for r in runs):
                continue
            kw = dict(sm, seed=1, nu_max=40, inner=inner, krylov=True, tol=1e-8, max_cycles=200)
            vx.zero_()
            vy.zero_()
            ctx.vcycle(vx, vy, None, **kw)  # builds the hierarchy and the graph
            vx.zero_()
            vy.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, e, cyc = ctx.vcycle(vx, vy, None, **kw)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            runs.append({"schedule": sm, "seconds": dt, "cycles": cyc, "final_energy_residual": e, "status": st})
        best = min(runs, key=lambda r: r["seconds"] if r["status"] == 0 else float("inf"))
        out[inner + "_inner"] = dict(best, schedule="ras %dx%d k%d o%d" % (best["schedule"]["tile"] + (
            best["schedule"]["k"], best["schedule"]["overlap"])))
        out[inner + "_tried"] = [["ras %dx%d k%d o%d" % (r["schedule"]["tile"] + (r["schedule"]["k"],
                                                                                 r["schedule"]["overlap"])),
                                  round(r["seconds"], 4), r["cycles"]] for r in runs]
    # FP64 defect correction around FP32 flexible CG (8 iterations per outer step)
    kw = dict(variant="ras", tile=(32, 32), k=4, overlap=3, seed=1, nu_max=40, inner="f32", krylov=2, inner_its=8,
              tol=1e-8, max_cycles=200)
    vx.zero_()
    vy.zero_()
    ctx.vcycle(vx, vy, None, **kw)
    vx.zero_()
    vy.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, e, cyc = ctx.vcycle(vx, vy, None, **kw)
    torch.cuda.synchronize()
    out["f32_inner_cg_refinement"] = {"seconds": time.perf_counter() - t0, "v_cycles": cyc,
                                      "final_energy_residual": e, "status": st,
                                      "schedule": "FP64 defect correction around 8 FP32 CG iterations, ras 32x32 k4 o3"}
    out["speedup_f32_over_f64"] = out["f64_inner"]["seconds"] / min(out["f32_inner"]["seconds"],
                                                                    out["f32_inner_cg_refinement"]["seconds"])
    ctx.close()
    return out


def batch_leg(args, api):
    """The batched workload: 256 seeded sinkers of uneven sizes (sides
    64..1024, contrasts 1e2..1e6), all advanced together by the batched path
    versus a loop over one context per instance.  Smoothing: FP32 RAS in the
    schedule the autotuner picked for this batch, 20 sweeps per call,
    aggregate Gcell-updates/s.  Solve:
    FP64 flexible CG around the FP32 V-cycle to E_v <= 1e-8 for every
    instance, wall time of the whole set (hierarchies and graphs built
    beforehand)."""
    import torch
    from paper_2509_19061_gb300 import inputs
    specs = inputs.batch_specs(seed=5, count=args.batch)
    probs = [inputs.batch_problem(sp) for sp in specs]
    cells = sum(q.nx * q.ny for q in probs)
    out = {"workload": "batch_%d_sinkers_64to1024_seed5" % len(probs), "instances": len(probs),
           "cells_total": cells}
    sw = 20
    from paper_2509_19061_gb300 import autotune
    tuned = autotune.Cache(autotune.SHIPPED).batch(autotune.BATCH_NAME if len(probs) == 256 else "")
    sched = dict(variant="ras", tile=(tuned.tile_i, tuned.tile_j), k=tuned.k, overlap=tuned.overlap, seed=1)
    label = "ras %dx%d k%d o%d (autotuned on this batch)" % (tuned.tile_i, tuned.tile_j, tuned.k, tuned.overlap)
    smooth_kw = dict(sched, sweeps=sw)
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps / 1e3

    # batched smoothing
    b = api.BatchContext([q.nx for q in probs], [q.ny for q in probs], dtype="f32")
    b.set_problems(probs)
    vx, vy = b.slab(), b.slab()
    k0 = b.kernels()
    t_b = timed(lambda: b.smooth(vx, vy, None, **smooth_kw), 5)
    launches_b = (b.kernels() - k0) // 6
    # one context per instance
    ctxs = []
    for q in probs:
        c = api.StokesContext(q.nx, q.ny, 1.0, 1.0, "f32")
        c.set_problem(q)
        ctxs.append((c, c.field(), c.field()))

    def loop():
        for c, x, y in ctxs:
            c.smooth(x, y, None, **smooth_kw)
    t_l = timed(loop, 2)
    for c, _, _ in ctxs:
        c.close()
    b.close()
    out["smooth"] = {"sweeps": sw, "schedule": label + " f32",
                     "batched_gcell_updates_per_s": cells * sw / t_b / 1e9, "batched_ms": 1e3 * t_b,
                     "batched_launches": launches_b,
                     "per_instance_gcell_updates_per_s": cells * sw / t_l / 1e9, "per_instance_ms": 1e3 * t_l,
                     "speedup": t_l / t_b}
    # time to E_v <= 1e-8 for every instance
    kw = dict(sched, nu_max=40, inner="f32", krylov=True, tol=1e-8, max_cycles=300)
    b = api.BatchContext([q.nx for q in probs], [q.ny for q in probs], dtype="f64")
    b.set_problems(probs)
    vx, vy = b.slab(), b.slab()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.solve(vx, vy, None, **kw)  # hierarchy, dense coarsest inverses, plans, graph, and one solve
    torch.cuda.synchronize()
    t_first = time.perf_counter() - t0
    vx.zero_()
    vy.zero_()
    torch.cuda.synchronize()
    k0 = b.kernels()
    t0 = time.perf_counter()
    st, e, cyc, sts = b.solve(vx, vy, None, **kw)
    torch.cuda.synchronize()
    t_bs = time.perf_counter() - t0
    kb = b.kernels() - k0
    b.close()
    t_ls, worst, conv = 0.0, 0, 0
    for q in probs:
        c = api.StokesContext(q.nx, q.ny, 1.0, 1.0, "f64")
        c.set_problem(q)
        x, y = c.field(), c.field()
        c.vcycle(x, y, None, **kw)
        x.zero_()
        y.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s1, e1, c1 = c.vcycle(x, y, None, **kw)
        torch.cuda.synchronize()
        t_ls += time.perf_counter() - t0
        worst = max(worst, c1)
        conv += s1 == api.STOKES_OK
        c.close()
    out["solve"] = {"tol": 1e-8, "outer": "f64 flexible CG", "inner": "f32 V-cycle, %s, nu cap 40" % label,
                    "batched_seconds": t_bs, "batched_first_call_seconds": t_first, "batched_status": int(st),
                    "batched_converged": int(sum(1 for x in sts if x == api.STOKES_OK)),
                    "batched_max_cycles": int(max(cyc)), "batched_kernels": int(kb),
                    "per_instance_seconds": t_ls, "per_instance_converged": int(conv),
                    "per_instance_max_cycles": int(worst), "speedup": t_ls / t_bs}
    return out


def uzawa_leg(args, api):
    """The full Stokes solve of Sec. 6.2 on the centred sinker (1024^2,
    contrast 1e6): inexact Uzawa with a velocity step of four CG iterations,
    each preconditioned by one V-cycle (RAS 32 x 32, k = 4, overlap 3; one
    step per cycle stalls at this size), omega_p = 0.6, lithostatic start,
    continuation in five stages of 25 cycles; wall time until the full
    relative energy residual (velocity and pressure) reaches 1e-8, with the
    V-cycle in FP32 or FP64 (outer iteration FP64)."""
    import torch
    from paper_2509_19061_gb300 import inputs
    n = args.uzawa_n
    prob = inputs.sinker_problem(n, eta_in=1e6)
    out = {"workload": "sinker_%dx%d_contrast1e6" % (n, n), "tol": 1e-8, "omega_p": 0.6,
           "continuation": "theta 0, 1/4, .., 1 every 25 cycles",
           "velocity_step": "4 CG iterations, each one V-cycle (ras 32x32 k4 o3)"}
    for inner, label, aa in (("f32", "f32_inner", 0), ("f64", "f64_inner", 0), ("f32", "f32_inner_anderson5", 5)):
        ctx = api.StokesContext(n, n, 1.0, 1.0, "f64")
        ctx.set_problem(prob)
        vx, vy, p = ctx.field(), ctx.field(), ctx.field()
        kw = dict(cycles=600, theta_interval=25, tol=1e-8, inner=inner, variant="ras", tile=(32, 32), k=4,
                  overlap=3, seed=1, nu_max=40, vel_its=4, anderson=aa)
        ctx.uzawa(vx, vy, p, **dict(kw, cycles=2))  # hierarchy and graph
        vx.zero_()
        vy.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, hist, cyc, e = ctx.uzawa(vx, vy, p, **kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[label] = {"seconds": dt, "cycles": cyc, "final_energy_residual": e, "status": st,
                                 "ms_per_cycle": 1e3 * dt / max(cyc, 1),
                                 "residual_at": {str(c): float(hist[c - 1]) for c in (25, 50, 100, 200, 400)
                                                 if c <= len(hist)}}
        ctx.close()
    out["speedup_f32_over_f64"] = out["f64_inner"]["seconds"] / out["f32_inner"]["seconds"]
    return out


def robustness_leg(args, api):
    """The smoother comparison of Sec. 6.3 / Fig. (convergence history): the
    centred sinker at the paper's contrast 1e8 (256^2), inexact Uzawa with
    continuation (five stages of 25 cycles), one CG step preconditioned by
    one V-cycle per cycle, omega_u = 0.3, omega_p = 0.6; smoothers RBGS,
    Jacobi, RAS (32 x 32 tiles, k = 4, overlap 0: the paper's ring-only tile)
    and mixed.  RAS and mixed draw their tile shifts from 10 seeds and the
    worst seed is reported, as the paper reports the worst of ten runs;
    Jacobi and RBGS are deterministic (one run)."""
    n = args.robust_n
    out = robustness_run(api, n, n, cycles=300, levels=16, nu_max=40)
    # the paper's multigrid schedule (Sec. 6.2): 4 levels, 5 sweeps times 2.5
    # per coarser level without a cap, 1000 cycles, a grid with hx != hy.  The
    # paper's 501 x 601 grid cannot be halved (odd sides); 160 x 192 on the
    # unit square keeps hx != hy and four halvings' coarsest level (20 x 24,
    # 916 unknowns) within the dense coarsest solve.
    out["paper_schedule"] = robustness_run(api, 160, 192, cycles=1000, levels=4, nu_max=0)
    # the same grid with the default hierarchy and eight CG steps (each one
    # V-cycle) per Uzawa cycle: one step is too inexact a velocity solve there
    out["hx_ne_hy_8_steps"] = robustness_run(api, 160, 192, cycles=300, levels=16, nu_max=40, vel_its=8)
    return out


def robustness_run(api, nx, ny, cycles, levels, nu_max, vel_its=1):
    import torch
    from paper_2509_19061_gb300 import inputs
    prob = inputs.sinker_problem(nx, ny, eta_in=1e8)
    ctx = api.StokesContext(nx, ny, 1.0, 1.0, "f64")
    ctx.set_problem(prob)
    vx, vy, p = ctx.field(), ctx.field(), ctx.field()
    marks = [c for c in (25, 50, 100, 150, 200, 300, 500, 750, 1000) if c <= cycles]
    out = {"workload": "sinker_%dx%d_contrast1e8" % (nx, ny), "cycles": cycles, "levels": levels,
           "sweeps": "5 x 2.5^level pre and post" + (", capped at %d" % nu_max if nu_max else ", uncapped"),
           "uzawa": "continuation 5 x 25 cycles, %d CG step(s) of one V-cycle per cycle, omega_p 0.6" % vel_its,
           "report": "worst seed: max over seeds of the residual at each mark; cycles to 1e-8 (-1: not reached)"}
    for name, sm, seeds in (("rbgs", dict(variant="rbgs"), [0]), ("jacobi", dict(variant="jacobi"), [0]),
                            ("ras", dict(variant="ras", tile=(32, 32), k=4, overlap=0), range(10)),
                            ("mixed", dict(variant="mixed", tile=(32, 32), k=4, overlap=0), range(10))):
        worst, reach, secs = None, [], 0.0
        for sd in seeds:
            vx.zero_()
            vy.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, hist, cyc, e = ctx.uzawa(vx, vy, p, cycles=cycles, theta_interval=25, inner="f32", nu_max=nu_max,
                                         levels=levels, seed=sd, vel_its=vel_its, **sm)
            torch.cuda.synchronize()
            secs += time.perf_counter() - t0
            h = np.asarray(hist)
            worst = h if worst is None else np.maximum(worst, h)
            hit = np.nonzero(h <= 1e-8)[0]
            reach.append(int(hit[0]) + 1 if len(hit) else -1)
        out[name] = {"seeds": len(list(seeds)),
                     "worst_residual_at": {str(c): float(worst[c - 1]) for c in marks if c <= len(worst)},
                     "cycles_to_1e-8": reach, "seconds_per_run": secs / len(list(seeds))}
    ctx.close()
    return out


def autotune_leg(args, api):
    """One tuning run of the RAS smoother (tile, k, overlap) by wall time of
    the solve to E_v <= 1e-8: 1024^2 centred sinker, contrast 1e4, FP64 outer
    flexible CG around the FP32 V-cycle, the tuner's default candidate list."""
    from paper_2509_19061_gb300 import autotune, inputs
    prob = inputs.sinker_problem(1024, eta_in=1e4)
    win, table = autotune.tune(api, prob, dtype="f64", inner="f32")
    dflt = [c for c in table if (c.tile_i, c.tile_j, c.k, c.overlap) == (32, 32, 4, 3)]
    return {"workload": "sinker_1024x1024_contrast1e4", "objective": "seconds to E_v <= 1e-8",
            "best": {"tile": [win.tile_i, win.tile_j], "k": win.k, "overlap": win.overlap,
                     "seconds": win.seconds, "cycles": win.cycles},
            "default_32x32_k4_o3_seconds": dflt[0].seconds if dflt else None,
            "candidates": [[c.tile_i, c.tile_j, c.k, c.overlap, round(c.seconds, 5), c.cycles] for c in table]}


def _time_smooth(ctx, vx, vy, kw, reps=2):
    import torch
    stream = torch.cuda.current_stream()
    ctx.smooth(vx, vy, None, **kw)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.smooth(vx, vy, None, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def energy_weights(prob):
    """-diag(M) at the velocity unknowns (zero elsewhere) in the natural
    layouts, from the viscosities of an inputs.Problem (eta_n zero on the
    boundary nodes: free slip)."""
    import numpy as np
    ec = np.asarray(prob.eta_c, dtype=np.float64)
    en = np.array(prob.eta_n, dtype=np.float64)
    en[0, :] = en[-1, :] = en[:, 0] = en[:, -1] = 0.0
    ihx2, ihy2 = 1.0 / prob.hx ** 2, 1.0 / prob.hy ** 2
    ny, nx = ec.shape
    wx = np.zeros((ny, nx + 1))
    wx[:, 1:nx] = 2.0 * (ec[:, 1:] + ec[:, :-1]) * ihx2 + (en[1:, 1:nx] + en[:-1, 1:nx]) * ihy2
    wy = np.zeros((ny + 1, nx))
    wy[1:ny, :] = 2.0 * (ec[1:, :] + ec[:-1, :]) * ihy2 + (en[1:ny, 1:] + en[1:ny, :-1]) * ihx2
    return wx, wy


def fp32_error_leg(args, api, prob):
    """The FP32 result of the benchmark's smoothing (100 sweeps from zero,
    the benchmark's schedule) against the FP64 GPU result of the same map
    (RAS with overlap k - 1 is exact Jacobi whatever the tiles; the FP64 path
    matches the FP64 oracle to 1e-12 in the tests), in the diag(-M)-weighted
    energy norm, relative."""
    import numpy as np
    n = args.n
    k = args.k
    o = args.overlap if args.overlap is not None else k - 1
    if o < k - 1:
        return {"skipped": "the schedule is not exact Jacobi"}
    res = {}
    for dt_name, kw in (("f32", dict(tile=tuple(args.tile), k=k, overlap=o)),
                        ("f64", dict(tile=(32, 32), k=4, overlap=3))):
        c = api.StokesContext(n, n, 1.0, 1.0, dt_name)
        c.set_problem(prob)
        vx, vy = c.field(), c.field()
        c.smooth(vx, vy, None, variant="ras", sweeps=args.sweeps, seed=7, **kw)
        res[dt_name] = (c.unpack(vx, "vx"), c.unpack(vy, "vy"))
        c.close()
    wx, wy = energy_weights(prob)
    (ax, ay), (bx, by) = res["f32"], res["f64"]
    num = np.sum(wx * (ax - bx) ** 2) + np.sum(wy * (ay - by) ** 2)
    den = np.sum(wx * bx ** 2) + np.sum(wy * by ** 2)
    return {"energy_norm_rel_error": float(np.sqrt(num / den)), "sweeps": args.sweeps,
            "fp32": "ras %dx%d k%d o%d" % (args.tile[0], args.tile[1], k, o),
            "fp64": "ras 32x32 k4 o3 (the same map: exact Jacobi)"}


def variant_table(args, api, prob):
    """The 8192^2 layered sinker (the throughput workload): FP32 and FP64
    RAS-Jacobi with k in {1, 2, 4, 8} (overlap k-1, exact Jacobi, and
    overlap 0, the paper's ring-only tile) and the other four smoothers.
    Gcell-updates/s and effective GB/s (8 words per cell-sweep) over the
    device time of the smoothing call; frac = effective GB/s over the
    measured HBM copy bandwidth."""
    n = args.n
    peak, _ = measured_peaks()
    out = {}
    cases = []
    for k in (1, 2, 4, 8):
        for o in sorted({k - 1, 0}):
            # 56 x 32 with overlap 7 is a 72-column window, wider than the packed-pair
            # layout's 64: the k = 8 exact row uses the 48 x 32 tile (a 64 x 48 window)
            tile = (48, 32) if (k == 8 and o == 7) else (56, 32)
            cases.append(("f32", dict(variant="ras", sweeps=40, tile=tile, k=k, overlap=o)))
    cases += [("f32", dict(variant="ras", sweeps=40, tile=(48, 32), k=8, overlap=7)),
              ("f32", dict(variant="ras", sweeps=40, tile=(48, 64), k=8, overlap=7)),
              ("f32", dict(variant="ras", sweeps=40, tile=(62, 32), k=8, overlap=0)),
              ("f32", dict(variant="ras", sweeps=40, tile=(62, 56), k=8, overlap=0)),
              ("f32", dict(variant="ras", sweeps=40, tile=(32, 32), k=4, overlap=3)),
              ("f32", dict(variant="jacobi", sweeps=20)), ("f32", dict(variant="fused", sweeps=20)),
              ("f32", dict(variant="blocked", sweeps=20, tile=(56, 32))), ("f32", dict(variant="rbgs", sweeps=20))]
    for k in (1, 2, 4, 8):
        # an FP64 32 x 32 tile with overlap 7 is a 48 x 48 window, beyond the register
        # layout's 512 threads: the k = 8 row uses 24 x 24 tiles (a 40 x 40 window)
        tile = (24, 24) if k == 8 else (32, 32)
        cases.append(("f64", dict(variant="ras", sweeps=8, tile=tile, k=k, overlap=k - 1)))
    cases += [("f64", dict(variant="ras", sweeps=8, tile=(32, 32), k=4, overlap=0)),
              ("f64", dict(variant="fused", sweeps=4)), ("f64", dict(variant="rbgs", sweeps=4))]
    ctxs = {}
    for dt_name, kw in cases:
        if dt_name not in ctxs:
            c = api.StokesContext(n, n, 1.0, 1.0, dt_name)
            c.set_problem(prob)
            ctxs[dt_name] = (c, c.field(), c.field())
        c, vx, vy = ctxs[dt_name]
        ms = _time_smooth(c, vx, vy, kw)
        label = "%s_%s" % (dt_name, kw["variant"])
        if kw["variant"] in ("ras", "blocked"):
            label += "_%dx%d" % kw["tile"]
        if kw["variant"] == "ras":
            label += "_k%d_o%d" % (kw["k"], kw["overlap"])
        cu = n * n * kw["sweeps"] / (ms / 1e3)
        gbs = cu * WORDS_PER_CELL_SWEEP * (8 if dt_name == "f64" else 4) / 1e9
        out[label] = {"gcell_updates_per_s": cu / 1e9, "effective_gbs": gbs, "frac": gbs / peak,
                      "sweeps": kw["sweeps"], "ms_per_call": ms}
        if kw["variant"] in ("ras", "blocked"):
            out[label]["kernel"] = tile_kernel_name(api, n, kw["tile"], kw.get("overlap", 0), dt_name)
    for c, _, _ in ctxs.values():
        c.close()
    return out


def smoothers_leg(args, api):
    """The global-memory smoothers (Jacobi as separate vx / vy passes, fused
    Jacobi, red-black Gauss-Seidel) on the layered sinker at --n, FP32 and
    FP64: one warm-up call and three timed calls of `sweeps` sweeps each
    (few launches, so that an ncu capture of the same command stays small).
    Gcell-updates/s and effective GB/s (8 words per cell-sweep) over the
    measured HBM copy bandwidth."""
    from paper_2509_19061_gb300 import inputs
    n = args.n
    peak, _ = measured_peaks()
    prob = inputs.layered_sinker(n, seed=4)
    out = {}
    for dt_name, sweeps in (("f32", 4), ("f64", 2)):
        c = api.StokesContext(n, n, 1.0, 1.0, dt_name)
        c.set_problem(prob)
        vx, vy = c.field(), c.field()
        for v in ("jacobi", "fused", "rbgs"):
            kw = dict(variant=v, sweeps=sweeps)
            ms = _time_smooth(c, vx, vy, kw, reps=3)
            cu = n * n * sweeps / (ms / 1e3)
            gbs = cu * WORDS_PER_CELL_SWEEP * (8 if dt_name == "f64" else 4) / 1e9
            out["%s_%s" % (dt_name, v)] = {"gcell_updates_per_s": cu / 1e9, "effective_gbs": gbs,
                                            "frac": gbs / peak, "sweeps": sweeps, "ms_per_call": ms}
        c.close()
    return out


def slabs_leg(args, api):
    """The slab decomposition of RAS (one slab per GPU in a multi-GPU run; here
    every slab on this GPU): the benchmark's smoothing (FP32 layered sinker at
    --n, RAS 48 x 64, k = 8, overlap 7, 100 sweeps) split into 2, 4 and 8 row
    slabs against one context.  Per slab count: the time of one smoothing call
    (CUDA events, one warm-up call first), Gcell-updates/s, the halo copies and
    bytes of one call, and whether the result equals the single context bit
    for bit."""
    import torch
    from paper_2509_19061_gb300 import inputs
    n, sweeps = args.n, 100
    kw = dict(variant="ras", sweeps=sweeps, tile=(48, 64), k=8, overlap=7, seed=1)
    prob = inputs.layered_sinker(n, seed=4)
    ctx = api.StokesContext(n, n, 1.0, 1.0, "f32")
    ctx.set_problem(prob)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ref = (ctx.field(), ctx.field())
    ctx.smooth(*ref, None, **kw)
    for v in ref:
        v.zero_()
    e0.record(stream)
    ctx.smooth(*ref, None, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out = {"workload": "layered_sinker_%dx%d_ras_f32_48x64_k8_o7_%dsweeps" % (n, n, sweeps),
           "single": {"ms_per_call": ms, "gcell_updates_per_s": n * n * sweeps / (ms / 1e3) / 1e9}}
    eta_c, eta_n = ctx.pack(prob.eta_c, "eta_c"), ctx.pack(prob.eta_n, "eta_n")
    fx, fy = ctx.pack(prob.fx, "fx"), ctx.pack(prob.fy, "fy")
    for ns in (2, 4, 8):
        sl = api.SlabContext(n, n, 1.0, 1.0, "f32", ns)
        sl.set_viscosity_dev(eta_c, eta_n)
        sl.set_rhs_dev(fx, fy)
        vx, vy = ctx.field(), ctx.field()
        sl.smooth(vx, vy, None, **kw)
        vx.zero_()
        vy.zero_()
        c0 = sl.exchanges()
        e0.record(stream)
        sl.smooth(vx, vy, None, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        c1 = sl.exchanges()
        out["slabs_%d" % ns] = {"ms_per_call": ms, "gcell_updates_per_s": n * n * sweeps / (ms / 1e3) / 1e9,
                                "halo_copies_per_call": c1[0] - c0[0], "halo_bytes_per_call": c1[1] - c0[1],
                                "bitwise_equal_single": bool(torch.equal(vx, ref[0]) and torch.equal(vy, ref[1]))}
        sl.close()
    ctx.close()
    return out


WORDS_PER_CELL_SWEEP_3D = 13  # read vx, vy, vz, eta_c, eta_xy, eta_xz, eta_yz, bx, by, bz; write vx, vy, vz


def smooth3d_leg(args, api):
    """The 3D operator (the 3D extension of Sec. 9): the layered 3D sinker at
    --n3d cells per side (fields of 4 or 8 bytes x (n+1)^2 x pitch, far above
    L2), FP32 and FP64: fused Jacobi and RAS-Jacobi on 3D tiles (space and
    time blocked together), one warm-up call, then three timed calls.
    Gcell-updates/s (one cell-update: its vx, vy and vz once) and effective
    GB/s at 13 words per cell-sweep over the measured HBM copy bandwidth."""
    from paper_2509_19061_gb300 import inputs
    peak, _ = measured_peaks()
    out = {}
    for dt_name, n in (("f32", args.n3d), ("f64", max(64, args.n3d // 2))):
        prob = inputs.layered3d_problem(n, seed=6)
        ctx = api.Stokes3DContext(n, n, n, 1.0, 1.0, 1.0, dt_name)
        ctx.set_problem(prob)
        v = [ctx.field() for _ in range(3)]
        # 8^3 tiles run the general tile kernel; windows 16 to 32 cells wide
        # (30 x 6 x 6 and 28 x 8 x 4 with one ring or overlap 1) the column kernel
        cases = [dict(variant="fused", sweeps=4), dict(variant="ras", sweeps=4, tile=(8, 8, 8), k=2, overlap=1),
                 dict(variant="ras", sweeps=4, tile=(8, 8, 8), k=4, overlap=0),
                 dict(variant="ras", sweeps=4, tile=(30, 6, 6), k=4, overlap=0),
                 dict(variant="ras", sweeps=4, tile=(28, 4, 4) if dt_name == "f64" else (28, 8, 4), k=2, overlap=1)]
        if dt_name == "f32":
            cases.append(dict(variant="ras", sweeps=8, tile=(30, 14, 6), k=8, overlap=0))
        import torch
        stream = torch.cuda.current_stream()
        for kw in cases:
            ctx.smooth(*v, None, **kw)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                ctx.smooth(*v, None, **kw)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 3
            cu = n ** 3 * kw["sweeps"] / (ms / 1e3)
            gbs = cu * WORDS_PER_CELL_SWEEP_3D * (8 if dt_name == "f64" else 4) / 1e9
            label = "%s_%d_%s" % (dt_name, n, kw["variant"])
            if kw["variant"] == "ras":
                label += "_%dx%dx%d_k%d_o%d" % (kw["tile"] + (kw["k"], kw["overlap"]))
            out[label] = {"gcell_updates_per_s": cu / 1e9, "effective_gbs": gbs, "frac": gbs / peak,
                          "ms_per_call": ms, "sweeps": kw["sweeps"]}
        e = ctx.energy(*v)
        out["%s_%d_energy_after" % (dt_name, n)] = (e[0] / e[2]) ** 0.5
        ctx.close()
    return out


def c2_table(args, api):
    """The 1024^2 sinker at contrast 1e4 in FP64: all five smoothers, 100
    sweeps each (--c2-sweeps), RAS with tiles 16^2, 32^2, 64 x 32 and k in {1, 2, 4, 8}
    (overlap k-1).  The FP64 working set (8 fields x 8.4 MB) fits in the
    129 MB L2, so these rates are L2-, not HBM-bound."""
    from paper_2509_19061_gb300 import inputs
    n = 1024
    prob = inputs.sinker_problem(n, eta_in=1e4)
    c = api.StokesContext(n, n, 1.0, 1.0, "f64")
    c.set_problem(prob)
    vx, vy = c.field(), c.field()
    sw = args.c2_sweeps
    cases = [dict(variant=v, sweeps=sw) for v in ("jacobi", "fused", "rbgs")]
    cases.append(dict(variant="blocked", sweeps=sw, tile=(32, 32)))
    for tile in ((16, 16), (32, 32), (64, 32), (24, 24)):
        for k in (1, 2, 4, 8):
            cases.append(dict(variant="ras", sweeps=sw, tile=tile, k=k, overlap=k - 1))
    out = {}
    for kw in cases:
        label = kw["variant"]
        if kw["variant"] in ("ras", "blocked"):
            label += "_%dx%d" % kw["tile"]
        if kw["variant"] == "ras":
            label += "_k%d" % kw["k"]
            plan = api.stokes_tile_kernel_plan(n, n, kw["tile"], kw["overlap"], "f64")
            if plan[0] == "shared":
                # the FP64 window exceeds the register layouts (more than 512 threads):
                # the general shared-memory kernel, not a schedule to run
                out[label] = {"skipped": "window %d x %d exceeds the FP64 register layouts" % (
                    kw["tile"][0] + 2 * kw["k"], kw["tile"][1] + 2 * kw["k"])}
                continue
        try:
            ms = _time_smooth(c, vx, vy, kw, reps=1)
        except api.StokesError as ex:
            # FP64 windows of large tiles and deep overlaps exceed shared memory
            out[label] = {"error": str(ex)}
            continue
        cu = n * n * kw["sweeps"] / (ms / 1e3)
        out[label] = {"gcell_updates_per_s": cu / 1e9, "effective_gbs": cu * WORDS_PER_CELL_SWEEP * 8 / 1e9,
                      "ms_per_call": ms, "sweeps": sw}
    c.close()
    return {"workload": "sinker_1024x1024_contrast1e4_f64", "table": out}


def run_only(args):
    import torch
    from paper_2509_19061_gb300 import api
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if args.only == "fp32err":
        from paper_2509_19061_gb300 import inputs
        print(json.dumps({"leg": args.only, "result": fp32_error_leg(args, api, inputs.layered_sinker(args.n, seed=4))}))
        return 0
    leg = {"solve": solve_times, "batch": batch_leg, "autotune": autotune_leg, "c2": c2_table,
           "uzawa": uzawa_leg, "robustness": robustness_leg, "smoothers": smoothers_leg,
           "smooth3d": smooth3d_leg, "slabs": slabs_leg}[args.only]
    print(json.dumps({"leg": args.only, "result": leg(args, api)}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
