#!/usr/bin/env python3
"""Benchmark of the propagator build + composition (one step = the whole path).

Default workload: periodic 2-D advection-diffusion u_t = 0.01 lap(u) -
(1, 0.5).grad(u) on a 64 x 64 grid (d = 4096), t in [0, 1], S = 512 slices,
RK4 with dt = 2e-4 (m = 10 steps per slice), exact affine slice maps from
d + 1 = 4097 basis solves (68.7 GB in float64), composed into the final state.
One step = build all maps (computation phase) + compose them from u0
(communication phase).

Prints ONE JSON line.  The headline is the float64 method; the float32 and
refined reduced-precision variants, their errors against the float64 oracle
and the time to solution at the plain method's error are listed beside it.
--workload heat1d runs the 1-D heat equation (n = 256, S = 1024) the same way;
the other workloads print their own lines.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nvpit|reference]
                  [--workload advdiff2d|heat1d|vdp_batch|scalar|chain3_mlp|wave|square]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# The oracle timed as the CPU baseline runs on one host thread: no BLAS thread
# pool behind numpy's products (set before numpy is first imported), so the
# "cores": 1 in the baseline objects is what it used.
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

METRIC = "propagator-build trajectory-steps/s + time-to-solution vs plain at fixed error"
UNIT = "trajectory-steps/s"
L2_FLUSH_BYTES = 256 << 20          # > 129 MB L2
FP64_PEAK_NOMINAL = 1.25e12          # FLOP/s, FMA = 2 (GB300 FP64)
FP32_PEAK_NOMINAL = 152 * 128 * 2 * 2.07e9
FLOP_PER_COMPONENT_STEP = 20         # Horner-form RK4 step of the 3-point stencil
FLOP_PER_ROW_STEP_POLY9 = 13         # the nine-point form executed: 4 DADD + 1 DMUL + 4 DFMA
def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 10 for advection-diffusion, whose float64 steps take about "
                         "3 s; 100 for the heat equation, whose steps take a few ms; else 20)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="nvpit", choices=["nvpit", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variants", default=None,
                    help="precisions timed beside the float64 headline; prec:p sets p correction passes "
                         "(default: fp32,fp32_refine,fp32_refine:2,bf16_refine for advection-diffusion, "
                         "fp32,tf32_refine,fp32_refine,fp32_refine:2 for the heat equation)")
    ap.add_argument("--slices", type=int, default=0, help="override S (profiling a reduced case)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-probe", action="store_true")
    ap.add_argument("--workload", default="advdiff2d",
                    choices=["advdiff2d", "heat1d", "vdp_batch", "scalar", "chain3_mlp", "wave", "square"],
                    help="advdiff2d (default line) | heat1d | vdp_batch | scalar | chain3_mlp | wave | square")
    ap.add_argument("--instances", type=int, default=0, help="vdp_batch: use the first N instances")
    ap.add_argument("--train-steps", type=int, default=0, help="chain3_mlp: total Adam steps (profiling)")
    ap.add_argument("--learned-counts", default="128,1024,4096,65536",
                    help="chain3_mlp: state counts of the equal-error comparison")
    return ap.parse_args()


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate_over_ranks(units_local: float, seconds_local: float):
    """Whole-job throughput of replicas: units summed over ranks divided by the
    slowest rank's time (max over ranks).  Uses torch.distributed when it is
    initialised (NCCL on GPUs, gloo in the CPU tests); returns
    (value, max_seconds, total_units)."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([seconds_local], dtype=torch.float64, device=dev)
        u = torch.tensor([units_local], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        return float(u.item()) / float(t.item()), float(t.item()), float(u.item())
    return units_local / seconds_local, seconds_local, units_local


def traj_steps(w, m):
    """Trajectory-steps of one build: every basis column of every slice, m steps."""
    return w.S * (w.dim + 1) * m


# --------------------------------------------------------------- oracle legs

def oracle_sample(w, m, budget_s=10.0, min_slices=4):
    """The FP64 oracle's map build timed on host cores over a bounded sample of
    slices (as many as fit in budget_s, at least min_slices)."""
    from oracle import nievergelt as nv
    fi, fh = nv.workload_rhs(w, True), nv.workload_rhs(w, False)
    t0 = time.perf_counter()
    done = 0
    while done < w.S and (done < min_slices or time.perf_counter() - t0 < budget_s):
        nv.build_affine_slice(fi, fh, "rk4", w.t0, w.T, w.S, m, w.dim, done)
        done += 1
    el = time.perf_counter() - t0
    return done, el


def _oracle_slices(job):
    """Pool task: the oracle's map build of the given slices (returns how many)."""
    from oracle import nievergelt as nv
    w, m, slices = job
    fi, fh = nv.workload_rhs(w, True), nv.workload_rhs(w, False)
    for j in slices:
        nv.build_affine_slice(fi, fh, "rk4", w.t0, w.T, w.S, m, w.dim, j)
    return len(slices)


def _oracle_ready(_):
    from oracle import nievergelt  # noqa: F401  (import cost outside the timed region)
    return os.getpid()


class OraclePool:
    """The oracle on every host core: one spawned process per core (spawn, so no
    process inherits a CUDA context), one BLAS thread each, slices dealt out."""

    def __init__(self, procs=None):
        import multiprocessing
        self.procs = procs or os.cpu_count() or 1
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        self.pool = multiprocessing.get_context("spawn").Pool(self.procs)
        self.pool.map(_oracle_ready, range(self.procs))

    def build(self, w, m, slices):
        """Build the given slices across the pool; returns (slices built, seconds)."""
        jobs = [(w, m, slices[i::self.procs]) for i in range(self.procs)]
        t0 = time.perf_counter()
        done = sum(self.pool.map(_oracle_slices, jobs))
        return done, time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_sample_parallel(w, m, per_slice_s, budget_s=10.0):
    """The oracle's map build on all host cores over a bounded sample of slices
    (about budget_s of wall time, given the single-core time per slice)."""
    pool = OraclePool()
    try:
        count = min(w.S, max(pool.procs, int(budget_s * pool.procs / max(per_slice_s, 1e-6))))
        count -= count % pool.procs if count >= pool.procs else 0
        done, el = pool.build(w, m, list(range(count)))
    finally:
        pool.close()
    return done, el, pool.procs


def oracle_serial(w, m):
    from oracle import nievergelt as nv
    t0 = time.perf_counter()
    y = nv.serial_fine(nv.workload_rhs(w, True), "rk4", w.t0, w.T, w.S, m, w.y0)
    return y, time.perf_counter() - t0


def run_reference(args):
    """--impl reference: the float64 oracle itself, timed as it stands on every
    host core (one spawned process each), on the same workload, metric, unit
    and config object as the GPU line; each step a bounded sample of it."""
    world, rank, _ = dist_info()
    if rank != 0:
        return 0
    import workloads
    from oracle import nievergelt as nv
    if args.workload not in ("advdiff2d", "heat1d"):
        print(json.dumps({"impl": "reference",
                          "unavailable": "the reference arm times the oracle on the advdiff2d and heat1d "
                                         "workloads only"}))
        return 0
    adv = args.workload == "advdiff2d"
    w = workloads.advdiff2d() if adv else workloads.heat1d()
    m = nv.workload_steps(w)
    pool = OraclePool()                            # every host core, one process each

    if adv:
        # per step: one sample of ADV_ORACLE_COLUMNS basis columns (+ the solve
        # from 0) of one slice per process
        def step(i):
            items = adv_oracle_items(w, pool.procs, i * pool.procs)
            jobs = [(w, m, items[k::pool.procs]) for k in range(pool.procs)]
            t0 = time.perf_counter()
            cols = sum(pool.pool.map(_oracle_adv_columns, jobs))
            return cols * m, time.perf_counter() - t0
        sample = (f"per step {pool.procs} samples of {ADV_ORACLE_COLUMNS} of the 4096 basis columns "
                  f"(+ the solve from 0) of slices spread over the {w.S}, one per process")
    else:
        per_step = 8 * pool.procs                  # slices per reference step (bounded sample)

        def step(i):
            done, el = pool.build(w, m, [(i * per_step + k) % w.S for k in range(per_step)])
            return done * (w.dim + 1) * m, el
        sample = (f"{per_step} of {w.S} slices' maps per step (257 RK4 basis solves of n=256 each), "
                  f"dealt over {pool.procs} processes")
    try:
        for i in range(args.warmup):
            step(i)
        res = [step(args.warmup + i) for i in range(args.steps)]
    finally:
        pool.close()
    units = sum(u for u, _ in res)
    el = sum(t for _, t in res)
    val = units / el
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(w, m, world),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------- clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
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
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- GPU legs

def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def time_variant(nvp, torch, w, prec, K, W, flush, stream):
    """W untimed steps, then K timed steps; L2 flushed (untimed) before each.
    Returns per-step build / compose / total device times in ms and the result."""
    r = nvp.rhs("heat1d", w.dim, w.params)
    smp = nvp.samples("affine")
    st = nvp.steps("rk4", w.dt, 0, prec)
    y0 = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
    yT = torch.empty_like(y0)
    with torch.cuda.stream(stream):
        maps = nvp.build_propagators(r, w.t0, w.T, w.S, smp, st, stream=stream)
        for _ in range(W):
            nvp.build_propagators(r, w.t0, w.T, w.S, smp, st, maps=maps, stream=stream)
            nvp.compose(maps, y0, yT, stream=stream)
        nvp.maps_check(maps, stream=stream)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
        for k in range(K):
            flush.zero_()
            ev[k][0].record(stream)
            nvp.build_propagators(r, w.t0, w.T, w.S, smp, st, maps=maps, stream=stream)
            ev[k][1].record(stream)
            nvp.compose(maps, y0, yT, stream=stream)
            ev[k][2].record(stream)
        stream.synchronize()
    nvp.maps_check(maps, stream=stream)
    build = [e[0].elapsed_time(e[1]) for e in ev]
    comp = [e[1].elapsed_time(e[2]) for e in ev]
    tot = [a + b for a, b in zip(build, comp)]
    info = nvp.maps_info(maps)
    maps.destroy()
    return {"build_ms": build, "compose_ms": comp, "step_ms": tot, "yT": yT.cpu().numpy(),
            "m": info.steps_per_slice, "work_per_slice": info.work_per_slice,
            "build_kernel": info.build_kernel.decode()}


def time_serial_gpu(nvp, torch, w, stream, reps=3):
    """The plain serial fine solve on the GPU (nv_serial_fine: one warp, all S m
    RK4 steps in sequence), the other reference the method is measured against."""
    r = nvp.rhs("heat1d", w.dim, w.params)
    st = nvp.steps("rk4", w.dt, 0, "fp64")
    y0 = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
    ys = torch.empty_like(y0)
    with torch.cuda.stream(stream):
        nvp.serial_fine(r, w.t0, w.T, w.S, st, y0, ys, stream=stream)      # warm-up
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        for _ in range(reps):
            nvp.serial_fine(r, w.t0, w.T, w.S, st, y0, ys, stream=stream)
        ev[1].record(stream)
        stream.synchronize()
    return ev[0].elapsed_time(ev[1]) / reps, ys.cpu().numpy()


def time_e2e(nvp, torch, w, K, W, stream):
    """End to end through nv_solve (allocates, builds, composes, frees) with
    pinned host buffers copied in and out every step."""
    r = nvp.rhs("heat1d", w.dim, w.params)
    smp = nvp.samples("affine")
    st = nvp.steps("rk4", w.dt, 0, "fp64")
    y0_h = torch.tensor(w.y0, dtype=torch.float64).pin_memory()
    yT_h = torch.empty_like(y0_h).pin_memory()
    y0_d = torch.empty(w.dim, dtype=torch.float64, device="cuda")
    yT_d = torch.empty_like(y0_d)
    times = []
    with torch.cuda.stream(stream):
        for k in range(W + K):
            stream.synchronize()
            t0 = time.perf_counter()
            y0_d.copy_(y0_h, non_blocking=True)
            nvp.solve(r, w.t0, w.T, w.S, smp, st, y0_d, yT_d, stream=stream)
            yT_h.copy_(yT_d, non_blocking=True)
            stream.synchronize()
            if k >= W:
                times.append(time.perf_counter() - t0)
    return times, y0_h.numel() * 8, yT_h.numel() * 8


def gpu_peak_probe(torch):
    """Library FP64/FP32 GEMM rates on this GPU (context for the ALU roofline)."""
    out = {}
    for name, dt, n in (("fp64_dgemm_tflops", torch.float64, 4096), ("fp32_sgemm_tflops", torch.float32, 8192)):
        a = torch.randn(n, n, dtype=dt, device="cuda")
        b = torch.randn(n, n, dtype=dt, device="cuda")
        if dt == torch.float32:
            prev = torch.backends.cuda.matmul.allow_tf32
            torch.backends.cuda.matmul.allow_tf32 = False
        for _ in range(2):
            torch.matmul(a, b)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record()
        for _ in range(reps):
            torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        out[name] = 2 * n ** 3 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12
        if dt == torch.float32:
            torch.backends.cuda.matmul.allow_tf32 = prev
        del a, b
    return out


# DRAM bytes (read + write) per unit of output from one ncu capture of each
# dominant kernel, scaled to the bench's launch by the units it writes (the
# captures ran smaller cases of the same kernels; see profiles/):
#   heat FP64 build (nine-point form), S = 512 capture: 207.06 MB for 131 072 columns
#   heat FP64 build (two-window form), full size: 475.35 MB for 262 144 columns
#   heat FP64 build (three-window form), full size: 475.15 MB for 262 144 columns
#   advection-diffusion FP32 build, S = 8 capture: 475.04 MB for 32 776 columns
#   advection-diffusion FP32 build with windows, S = 8 capture: 475.46 MB for 32 776 columns
#   Van der Pol batch build, 512 instances: 503.0 MB for 561 987 584 table bytes
#   chain pairs, the full launch: 341.2 MB for 402 653 184 pair bytes
#   wave FP64 build, full size: 42.78 MB for 81 408 columns (maps fit in L2)
#   advection-diffusion FP32 chain, S = 8: 547.9 MB for 8 slice maps (537.0 MB read once)
#   advection-diffusion FP64 build (windows + row ladder), the full launch: 69.293 GB for 2 097 664 columns
NCU_TRAFFIC_PER_UNIT = {
    "affine_chain_tile_kernel<float,float>": (547.89e6 / 8, "profiles/advdiff_chains_d4096_S512.md"),
    "wave_build_kernel<double,80,2>": (42.78e6 / 81408, "profiles/wave_leapfrog_build_M80_S512.md"),
    "heat_poly9_kernel<double,8,0>": (207.06e6 / 131072, "profiles/heat_affine_build_and_chain_n256_S1024.md"),
    "heat_window2_kernel<double,4,11,0>": (475.35e6 / 262144, "profiles/heat_affine_build_and_chain_n256_S1024.md"),
    "heat_window3_kernel<double,2,11,0>": (475.15e6 / 262144, "profiles/heat_affine_build_and_chain_n256_S1024.md"),
    "advdiff_block_kernel<float>": (475.04e6 / 32776, "profiles/advdiff_fp32_block_build_64x64.md"),
    "advdiff_window_kernel<float>": (475.46e6 / 32776, "profiles/advdiff_fp32_block_build_64x64.md"),
    "advdiff_window64_kernel<16>": (69.293e9 / (512 * 4097), "profiles/advdiff_fp64_window_build_d4096_S512.md"),
    "batch_build_kernel<RhsVdp<float>,float,4,1>": (503.0e6 / 561987584, "profiles/vdp_batch_build_4096_instances.md"),
    "pairs_kernel<float>": (341.2e6 / 402653184, "profiles/chain3_pairs_build_S128_M65536.md"),
}


def ncu_traffic(kernel, units):
    per, src = NCU_TRAFFIC_PER_UNIT[kernel]
    return per * units, src


FP32_FLOP_PER_VDP_STEP = 52   # RK4 step of the 2-D Van der Pol system incl. compensated update


def _device_setup():
    import torch
    world, rank, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1304_6514_gb300 import _build
    _build.build()
    return torch, world, rank, local


def _max_over_ranks(torch, world, x):
    if world > 1:
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())
    return x


def run_vdp_batch(args):
    """4096 independent Van der Pol instances with uneven horizons and slice
    counts: one persistent build launch (LPT work queue) + float64 composition,
    replayed from a CUDA graph; CTA shape picked by the autotuner."""
    torch, world, rank, local = _device_setup()
    import numpy as np
    import paper_1304_6514_gb300 as nvp
    import workloads
    vb = workloads.vdp_batch()
    if args.instances > 0:
        k = args.instances
        vb = workloads.VdpBatch(vb.mu[:k], vb.T[:k], vb.S[:k], vb.y0[:k])
    P = vb.per_dim
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    smp = nvp.samples("bilinear2d", P, (vb.lo, vb.lo), (vb.hi, vb.hi))
    st = nvp.steps("rk4", vb.dt, 0, "fp32")
    K, W = args.steps, max(3, args.warmup)
    with torch.cuda.stream(stream):
        b = nvp.build_batch("vdp", 2, vb.mu, np.zeros_like(vb.T), vb.T, vb.S, smp, st, stream=stream)
        best = nvp.batch_autotune(b, stream=stream)
        info = nvp.batch_info(b)
        y0 = torch.tensor(vb.y0, dtype=torch.float64, device="cuda")
        yT = torch.empty_like(y0)
        for _ in range(W):
            nvp.batch_run(b, y0, yT, stream=stream)
        nvp.batch_check(b, stream=stream)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
        sampler = ClockSampler(local)
        sampler.start()
        for k in range(K):
            flush.zero_()
            ev[k][0].record(stream)
            nvp.batch_rebuild(b, stream=stream)
            ev[k][1].record(stream)
            nvp.batch_compose(b, y0, yT, stream=stream)
            ev[k][2].record(stream)
        gev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        gev[0].record(stream)
        for k in range(K):
            nvp.batch_run(b, y0, yT, stream=stream)
        gev[1].record(stream)
        stream.synchronize()
        clocks = sampler.stop()
        oob = nvp.batch_check(b, stream=stream)
    build = [e[0].elapsed_time(e[1]) for e in ev]
    comp = [e[1].elapsed_time(e[2]) for e in ev]
    step_s = _max_over_ranks(torch, world, sum(build) * 1e-3 + sum(comp) * 1e-3)
    graph_ms = gev[0].elapsed_time(gev[1]) / K
    units = info["traj_steps"]
    # the plain method on the same instances, one at a time: build + compose
    # per instance through the single-problem API (same tables, precision and
    # composition), timed on a sample of instances spread over the batch and
    # scaled by their share of the trajectory-steps
    yT_b = yT.cpu().numpy()
    pick = np.linspace(0, len(vb.mu) - 1, min(64, len(vb.mu))).astype(int)
    plain_ms, plain_units, plain_diff = 0.0, 0, 0.0
    with torch.cuda.stream(stream):
        y1 = torch.empty(2, dtype=torch.float64, device="cuda")
        yo = torch.empty_like(y1)
        for i in pick:
            r1 = nvp.rhs("vdp", 2, (float(vb.mu[i]),))
            y1.copy_(torch.tensor(vb.y0[i], dtype=torch.float64))
            mp = nvp.build_propagators(r1, 0.0, float(vb.T[i]), int(vb.S[i]), smp, st, stream=stream)
            nvp.compose(mp, y1, yo, stream=stream)                           # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            nvp.build_propagators(r1, 0.0, float(vb.T[i]), int(vb.S[i]), smp, st, maps=mp, stream=stream)
            nvp.compose(mp, y1, yo, stream=stream)
            e1.record(stream)
            stream.synchronize()
            plain_ms += e0.elapsed_time(e1)
            plain_units += int(vb.S[i]) * nvp.maps_info(mp).steps_per_slice * P * P
            plain_diff = max(plain_diff, float(np.abs(yo.cpu().numpy() - yT_b[i]).max()))
            mp.destroy()
    plain_total_ms = plain_ms * units / plain_units
    bmean = statistics.mean(build) * 1e-3
    achieved = FP32_FLOP_PER_VDP_STEP * units / bmean
    line = {"metric": METRIC, "value": units * K * world / step_s, "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": step_s / K * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 build, f64 composition",
            "data": "synthetic",
            "config": {"workload": "vdp_batch_4096_rk4_bilinear32", "instances": len(vb.mu),
                       "total_slices": info["total_slices"], "table_bytes": info["table_bytes"],
                       "cta_threads_autotuned": best, "l2": "flushed before every timed step"},
            "build_ms": statistics.mean(build), "compose_ms": statistics.mean(comp),
            "graph_run_ms": graph_ms, "out_of_range_evaluations": oob,
            "plain_per_instance": {"ms_for_all_instances": plain_total_ms,
                                   "speedup_of_batched_graph": plain_total_ms / graph_ms,
                                   "sample": f"{len(pick)} instances timed one by one, scaled by trajectory-steps",
                                   "max_abs_diff_vs_batched": plain_diff},
            "roofline": {"bound": "alu", "kernel": "batch_build_kernel<RhsVdp<float>,float,4,1>",
                         "achieved": achieved / 1e12, "peak": FP32_PEAK_NOMINAL / 1e12, "unit": "TFLOP/s",
                         "frac": achieved / FP32_PEAK_NOMINAL,
                         "traffic": ncu_traffic("batch_build_kernel<RhsVdp<float>,float,4,1>",
                                                info["table_bytes"])[0],
                         "traffic_source": ncu_traffic("batch_build_kernel<RhsVdp<float>,float,4,1>", 1)[1],
                         "algorithmic_bytes": info["table_bytes"],
                         "peak_source": "nominal FP32 (152 SMs x 128 lanes x 2 x 2.07 GHz)"},
            "gpu_launches": 2 * K, "clocks": clocks}
    # the same batch with float64 tables: the float32 final states' error
    # against the float64 method over all instances
    with torch.cuda.stream(stream):
        b64 = nvp.build_batch("vdp", 2, vb.mu, np.zeros_like(vb.T), vb.T, vb.S, smp,
                              nvp.steps("rk4", vb.dt, 0, "fp64"), stream=stream)
        yT64 = torch.empty_like(y0)
        nvp.batch_compose(b64, y0, yT64, stream=stream)
        nvp.batch_check(b64, stream=stream)
        b64.destroy()
    y64 = yT64.cpu().numpy()
    e32 = np.linalg.norm(yT_b - y64, axis=1) / np.maximum(np.linalg.norm(y64, axis=1), 1e-300)
    line["fp32_final_state_rel_err_vs_fp64_gpu"] = {
        "max": float(e32.max()), "median": float(np.median(e32)),
        "instances_above_1e-5": int(np.sum(e32 > 1e-5)), "instances": int(len(e32))}
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import nievergelt as nv
        # the oracle (float64 tables, float64 composition) on the instances the
        # parity test checks: cheap ones, the longest horizon, the most slices,
        # the largest damping (out-of-range lookups), the most steps per slice
        mstep = np.ceil(vb.T / vb.S / vb.dt - 1e-9)
        pick = list(np.argsort(vb.T)[:3]) + [int(np.argmax(vb.T)), int(np.argmax(vb.S)),
                                             int(np.argmax(vb.mu))] + list(np.argsort(-mstep)[:2])
        pick = list(dict.fromkeys(int(i) for i in pick))
        nodes = nv.uniform_nodes(vb.lo, vb.hi, P)
        errs32, errs64 = {}, {}
        for i in pick:
            mi = nv.steps_per_slice(0.0, vb.T[i], int(vb.S[i]), vb.dt)
            tab = nv.build_table_2d(nv.rhs_vdp(vb.mu[i]), "rk4", 0.0, vb.T[i], int(vb.S[i]), mi, nodes, nodes)
            lam, _ = nv.compose_tables_2d(vb.lo, vb.hi, tab, vb.y0[i])
            errs32[i] = float(np.linalg.norm(yT_b[i] - lam[-1]) / np.linalg.norm(lam[-1]))
            errs64[i] = float(np.linalg.norm(y64[i] - lam[-1]) / np.linalg.norm(lam[-1]))
        line["final_state_rel_err_vs_oracle"] = {
            "instances": pick, "fp32": errs32, "fp64": errs64,
            "fp32_max": max(errs32.values()), "fp64_max": max(errs64.values())}
        i = int(np.argmin(vb.T))
        t0 = time.perf_counter()
        m = nv.steps_per_slice(0.0, vb.T[i], int(vb.S[i]), vb.dt)
        nodes = nv.uniform_nodes(vb.lo, vb.hi, P)
        nv.build_table_2d(nv.rhs_vdp(vb.mu[i]), "rk4", 0.0, vb.T[i], int(vb.S[i]), m, nodes, nodes)
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": int(vb.S[i]) * m * P * P / el, "unit": UNIT, "cores": 1,
                                "kind": "oracle", "sample": f"tables of instance {i} ({el:.1f} s)"}
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_scalar(args):
    """y' = cos(t) y - y^3, S = 16, M = 64, 10^4 Euler steps per slice, float64:
    time to solution of the method against the serial fine solve on the GPU."""
    torch, world, rank, local = _device_setup()
    import numpy as np
    import paper_1304_6514_gb300 as nvp
    import workloads
    w = workloads.scalar_cos_cubic()
    stream = torch.cuda.Stream()
    r = nvp.rhs("cos_cubic", 1)
    smp = nvp.samples("pl1d", w.per_dim, w.lo, w.hi)
    st = nvp.steps("euler", 0.0, w.steps_per_slice, "fp64")
    K, W = args.steps, max(3, args.warmup)
    y0 = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
    yT = torch.empty_like(y0)
    ys = torch.empty_like(y0)
    with torch.cuda.stream(stream):
        maps = nvp.build_propagators(r, w.t0, w.T, w.S, smp, st, stream=stream)
        for _ in range(W):
            nvp.build_propagators(r, w.t0, w.T, w.S, smp, st, maps=maps, stream=stream)
            nvp.compose(maps, y0, yT, stream=stream)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
        for k in range(K):
            ev[k][0].record(stream)
            nvp.build_propagators(r, w.t0, w.T, w.S, smp, st, maps=maps, stream=stream)
            ev[k][1].record(stream)
            nvp.compose(maps, y0, yT, stream=stream)
            ev[k][2].record(stream)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        nvp.serial_fine(r, w.t0, w.T, w.S, st, y0, ys, stream=stream)
        s1.record(stream)
        stream.synchronize()
        nvp.maps_check(maps, stream=stream)
    build = [e[0].elapsed_time(e[1]) for e in ev]
    comp = [e[1].elapsed_time(e[2]) for e in ev]
    step_ms = statistics.mean([a + b for a, b in zip(build, comp)])
    units = w.S * w.per_dim * w.steps_per_slice
    line = {"metric": METRIC, "value": units / (step_ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "S": w.S, "M": w.per_dim, "steps_per_slice": w.steps_per_slice},
            "build_ms": statistics.mean(build), "compose_ms": statistics.mean(comp),
            "serial_fine_gpu_ms": s0.elapsed_time(s1),
            "speedup_vs_serial_fine_gpu": s0.elapsed_time(s1) / step_ms,
            "method_minus_serial": float(yT.item() - ys.item()),
            "roofline": {"bound": "latency",
                         "note": "1024 independent chains of 10^4 dependent FP64 steps: fewer chains "
                                 "than lanes; time per step is the dependent-latency floor"}}
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import nievergelt as nv
        t0 = time.perf_counter()
        nv.build_table_1d(nv.rhs_cos_cubic(), "euler", w.t0, w.T, 2, w.steps_per_slice,
                          nv.uniform_nodes(w.lo[0], w.hi[0], w.per_dim))
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 2 * w.per_dim * w.steps_per_slice / el, "unit": UNIT,
                                "cores": 1, "kind": "oracle", "sample": f"2 of {w.S} slices ({el:.1f} s)"}
    if rank == 0:
        print(json.dumps(line))
    return 0


FLOP_PER_ADV_COMPONENT_STEP = 40   # Horner RK4: 4 stages x 5 FMA (FMA = 2), what the kernels execute
SURVEY_FLOP_PER_ADV_COMPONENT_STEP = 68   # the literal four-stage form's count (k_i = L y + 3 updates)
ADV_TARGET = {"fp64": 1e-11, "fp32": 1e-5, "fp32_refine": 1e-5, "bf16_refine": 1e-4}


def bench_config(w, m, world):
    """The config object both arms print for a workload (identical dicts)."""
    cfg = {"workload": w.name, "n": w.dim, "S": w.S, "steps_per_slice": m,
           "basis_columns_per_slice": w.dim + 1, "t": [w.t0, w.T], "dt": w.dt,
           "parallelism": "replicas" if world > 1 else "single GPU"}
    if w.rhs == "advdiff2d":
        cfg["l2"] = "inputs larger than L2: every step writes and reads the maps (68.7 GB FP64)"
    else:
        cfg["l2"] = "flushed (256 MB write) before every timed step"
    return cfg


def adv_time(nvp, torch, w, prec, K, W, stream, passes=0, sampler=None, barrier=None):
    """W untimed + K timed steps (build all maps, then compose them from u0) of
    the advection-diffusion problem at one precision; CUDA events on the
    launching stream.  The first build allocates the maps and counts as a
    warm-up step."""
    r = nvp.rhs("advdiff2d", w.dim, w.params[:3])
    smp = nvp.samples("affine")
    st = nvp.steps("rk4", w.dt, 0, prec)
    y0 = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
    yT = torch.empty_like(y0)
    nvp.tune_set(5, passes)
    clocks, wall = None, None
    try:
        with torch.cuda.stream(stream):
            maps = nvp.build_propagators(r, w.t0, w.T, w.S, smp, st, stream=stream)
            nvp.compose(maps, y0, yT, stream=stream)
            for _ in range(max(0, W - 1)):
                nvp.build_propagators(r, w.t0, w.T, w.S, smp, st, maps=maps, stream=stream)
                nvp.compose(maps, y0, yT, stream=stream)
            nvp.maps_check(maps, stream=stream)
            ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
            if barrier:
                barrier()
            if sampler:
                sampler.start()
            wall0 = time.perf_counter()
            for k in range(K):
                ev[k][0].record(stream)
                nvp.build_propagators(r, w.t0, w.T, w.S, smp, st, maps=maps, stream=stream)
                ev[k][1].record(stream)
                nvp.compose(maps, y0, yT, stream=stream)
                ev[k][2].record(stream)
            stream.synchronize()
            if barrier:
                barrier()
            wall = time.perf_counter() - wall0
            if sampler:
                clocks = sampler.stop()
            nvp.maps_check(maps, stream=stream)
        info = nvp.maps_info(maps)
        maps.destroy()
    finally:
        nvp.tune_set(5, 0)
    torch.cuda.empty_cache()
    build = [e[0].elapsed_time(e[1]) for e in ev]
    comp = [e[1].elapsed_time(e[2]) for e in ev]
    return {"build_ms": build, "compose_ms": comp, "step_ms": [a + b for a, b in zip(build, comp)],
            "yT": yT.cpu().numpy(), "m": info.steps_per_slice, "work_per_slice": info.work_per_slice,
            "build_kernel": info.build_kernel.decode(), "map_bytes": info.bytes,
            "clocks": clocks, "wall_s": wall}


def adv_e2e(nvp, torch, w, K, W, stream, reuse=False):
    """End to end with pinned host buffers copied in and out every step.
    reuse=False: through nv_solve (allocates the 68.7 GB of float64 maps,
    builds, composes, frees).  reuse=True: nv_build_propagators into a maps
    object allocated once before the timed steps, then nv_compose, as a caller
    solving repeatedly would; every step still builds all maps and composes."""
    r = nvp.rhs("advdiff2d", w.dim, w.params[:3])
    smp = nvp.samples("affine")
    st = nvp.steps("rk4", w.dt, 0, "fp64")
    y0_h = torch.tensor(w.y0, dtype=torch.float64).pin_memory()
    yT_h = torch.empty_like(y0_h).pin_memory()
    y0_d = torch.empty(w.dim, dtype=torch.float64, device="cuda")
    yT_d = torch.empty_like(y0_d)
    maps = None
    times = []
    with torch.cuda.stream(stream):
        if reuse:
            maps = nvp.build_propagators(r, w.t0, w.T, w.S, smp, st, stream=stream)
        for k in range(W + K):
            stream.synchronize()
            t0 = time.perf_counter()
            y0_d.copy_(y0_h, non_blocking=True)
            if reuse:
                nvp.build_propagators(r, w.t0, w.T, w.S, smp, st, maps=maps, stream=stream)
                nvp.compose(maps, y0_d, yT_d, stream=stream)
            else:
                nvp.solve(r, w.t0, w.T, w.S, smp, st, y0_d, yT_d, stream=stream)
            yT_h.copy_(yT_d, non_blocking=True)
            stream.synchronize()
            if k >= W:
                times.append(time.perf_counter() - t0)
    if maps is not None:
        nvp.maps_check(maps)
        maps.destroy()
    return times, y0_h.numel() * 8, yT_h.numel() * 8, yT_h.numpy().copy()


def _oracle_adv_columns(job):
    """Pool task: the oracle's map build of the given (slice, columns) samples."""
    from oracle import nievergelt as nv
    w, m, items = job
    fi, fh = nv.workload_rhs(w, True), nv.workload_rhs(w, False)
    done = 0
    for j, cols in items:
        nv.build_affine_slice(fi, fh, "rk4", w.t0, w.T, w.S, m, w.dim, j, columns=cols)
        done += len(cols) + 1                     # + the solve from 0 (b_j)
    return done


ADV_ORACLE_COLUMNS = 128     # basis columns per oracle sample (plus the solve from 0)


def adv_oracle_items(w, count, offset=0):
    """`count` samples of ADV_ORACLE_COLUMNS basis columns, spread over slices
    and over the grid (column c = 1 + (k * 29 + j) mod d)."""
    import numpy as np
    items = []
    for i in range(offset, offset + count):
        j = (i * 37) % w.S
        cols = (np.arange(ADV_ORACLE_COLUMNS) * 29 + i * 7) % w.dim
        items.append((j, cols))
    return items


def adv_cpu_baseline(w, m, budget_s=10.0):
    """The float64 oracle's map build on the host: one core, then every core
    (one spawned process each), each a bounded sample of columns of slices."""
    from oracle import nievergelt as nv
    fi, fh = nv.workload_rhs(w, True), nv.workload_rhs(w, False)
    t0 = time.perf_counter()
    one, k = 0, 0
    while k < 2 or time.perf_counter() - t0 < budget_s:
        (j, cols), = adv_oracle_items(w, 1, k)
        nv.build_affine_slice(fi, fh, "rk4", w.t0, w.T, w.S, m, w.dim, j, columns=cols)
        one += len(cols) + 1
        k += 1
    el1 = time.perf_counter() - t0
    per_item = el1 / k
    pool = OraclePool()
    try:
        # processes sharing the host's memory bandwidth run each sample about
        # three times slower than one process alone
        n_items = max(pool.procs, int(budget_s / (3.0 * per_item)) * pool.procs)
        items = adv_oracle_items(w, n_items)
        jobs = [(w, m, items[i::pool.procs]) for i in range(pool.procs)]
        t1 = time.perf_counter()
        cols_done = sum(pool.pool.map(_oracle_adv_columns, jobs))
        elp = time.perf_counter() - t1
    finally:
        pool.close()
    return {"single": (one * m, el1, k), "parallel": (cols_done * m, elp, n_items), "procs": pool.procs}


def run_advdiff(args):
    """The default line: periodic 2-D advection-diffusion, 64 x 64 grid (d =
    4096), S = 512, RK4 dt = 2e-4 (m = 10): the float64 method (68.7 GB of
    maps, built then composed by the HBM-bound chain) as the headline, the
    float32 / refined / bfloat16 variants beside it with their errors against
    the float64 oracle."""
    torch, world, rank, local = _device_setup()
    import numpy as np
    import paper_1304_6514_gb300 as nvp
    import workloads
    w = workloads.advdiff2d(S=args.slices, T=args.slices / 512) if args.slices > 0 else workloads.advdiff2d()
    stream = torch.cuda.Stream()
    peaks, peaks_src = read_peaks()
    K, W = max(1, args.steps), max(3, args.warmup)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # the float64 pipe's measured FMA rate (before the timed region)
    fp64_rate = nvp.alu_rate("fp64", stream=stream)
    fp32_rate = nvp.alu_rate("fp32", stream=stream)

    # ---- headline: the float64 method
    res = adv_time(nvp, torch, w, "fp64", K, W, stream, sampler=ClockSampler(local), barrier=barrier)
    m = res["m"]
    units = traj_steps(w, m)
    value, dev_s, _ = aggregate_over_ranks(units * K, sum(res["step_ms"]) * 1e-3)
    build_s = statistics.mean(res["build_ms"]) * 1e-3
    comp_s = statistics.mean(res["compose_ms"]) * 1e-3
    point_steps = w.S * res["work_per_slice"]
    flop = FLOP_PER_ADV_COMPONENT_STEP * point_steps
    achieved = flop / build_s

    # ---- variants on the same workload
    variants = {}
    results = {"fp64": res["yT"]}
    for v in [x for x in args.variants.split(",") if x]:
        prec, _, passes = v.partition(":")
        try:
            rv = adv_time(nvp, torch, w, prec, K, W, stream, passes=int(passes) if passes else 0)
        except nvp.NvError as e:
            variants[v] = {"unavailable": str(e)}
            continue
        results[v] = rv["yT"]
        bs = statistics.mean(rv["build_ms"]) * 1e-3
        cs = statistics.mean(rv["compose_ms"]) * 1e-3
        vflop = FLOP_PER_ADV_COMPONENT_STEP * w.S * rv["work_per_slice"]
        variants[v] = {"ms_per_step": statistics.mean(rv["step_ms"]), "build_ms": bs * 1e3,
                       "compose_ms": cs * 1e3, "traj_steps_per_s": units / (bs + cs),
                       "build_kernel": rv["build_kernel"], "map_bytes": rv["map_bytes"],
                       "build_tflops": vflop / bs / 1e12,
                       "build_frac_of_measured_fp32": vflop / bs / fp32_rate,
                       "speedup_vs_fp64_plain": (build_s + comp_s) / (bs + cs)}
        if prec == "fp32":
            variants[v]["chain_hbm_gbs"] = rv["map_bytes"] / cs / 1e9
            variants[v]["chain_frac_of_hbm"] = rv["map_bytes"] / cs / 1e9 / peaks["hbm_gbs"]
        else:
            variants[v]["passes"] = int(passes) if passes else ("library default" if prec == "bf16_refine" else 1)
        ref = results["fp64"]
        variants[v]["rel_err_vs_fp64_gpu"] = float(np.linalg.norm(rv["yT"] - ref) / np.linalg.norm(ref))

    # ---- end to end through the one-call API with host buffers
    if args.no_e2e:
        e2e_t, h2d, d2h, e2e_y = [float("nan")], 0, 0, None
        solve_t, solve_y = [float("nan")], None
    else:
        e2e_t, h2d, d2h, e2e_y = adv_e2e(nvp, torch, w, 3, 1, stream, reuse=True)
        solve_t, _, _, solve_y = adv_e2e(nvp, torch, w, 3, 1, stream)
    # ---- the plain serial fine solve on the GPU (one CTA, all S m RK4 steps)
    r = nvp.rhs("advdiff2d", w.dim, w.params[:3])
    y0 = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
    ys = torch.empty_like(y0)
    with torch.cuda.stream(stream):
        st64 = nvp.steps("rk4", w.dt, 0, "fp64")
        nvp.serial_fine(r, w.t0, w.T, w.S, st64, y0, ys, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nvp.serial_fine(r, w.t0, w.T, w.S, st64, y0, ys, stream=stream)
        e1.record(stream)
        stream.synchronize()
    serial_ms = e0.elapsed_time(e1)
    serial_gpu = ys.cpu().numpy()
    peaks_probe = {} if args.no_probe else gpu_peak_probe(torch)

    tts = {"fp64": (build_s + comp_s) * 1e3}
    tts.update({k: v["ms_per_step"] for k, v in variants.items() if "ms_per_step" in v})
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": statistics.mean(res["step_ms"]), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(w, m, world),
        "time_to_solution_ms": tts,
        "fp64": {"build_ms": build_s * 1e3, "compose_ms": comp_s * 1e3, "map_bytes": res["map_bytes"],
                 "chain_hbm_gbs": res["map_bytes"] / comp_s / 1e9,
                 "chain_frac_of_hbm": res["map_bytes"] / comp_s / 1e9 / peaks["hbm_gbs"]},
        "serial_fine_gpu": {"ms": serial_ms,
                            "rel_diff_method": float(np.linalg.norm(res["yT"] - serial_gpu) / np.linalg.norm(serial_gpu)),
                            "note": "one CTA stepping all S m RK4 steps in sequence: the plain solve the "
                                    "method parallelises (the method does (d+1) times its work)"},
        "wall_s_timed_region": res["wall_s"],
        "roofline": {"bound": "alu", "kernel": res["build_kernel"],
                     "achieved": achieved / 1e12, "peak": fp64_rate / 1e12, "unit": "TFLOP/s",
                     "frac": achieved / fp64_rate,
                     "peak_source": "measured in this run: nv_alu_rate, FP64 FMA chains on every SM "
                                    "(nominal 1.25 TFLOP/s beside it)",
                     "frac_of_nominal": achieved / FP64_PEAK_NOMINAL,
                     "flop_per_unit": "40 per point-step: the Horner-form RK4 step, 4 stages x 5 DFMA, "
                                      "the float64 instructions the kernel executes",
                     "points_note": ("the build integrates each column's first min(m, 3) steps on a 32 x 32 "
                                     "window around its unit point and the next two on the 48 rows they can "
                                     "reach (exactly zero outside), the rest on the 64 x 64 grid; the FLOPs "
                                     "count the points integrated"),
                     "full_grid_equivalent_tflops": FLOP_PER_ADV_COMPONENT_STEP * units * w.dim / build_s / 1e12,
                     "survey_unit_tflops": SURVEY_FLOP_PER_ADV_COMPONENT_STEP * point_steps / build_s / 1e12,
                     "survey_unit_note": "68 FLOP per point-step (the four literal stages), for comparison",
                     "traffic": (ncu_traffic(res["build_kernel"], w.S * (w.dim + 1))[0]
                                 if res["build_kernel"] in NCU_TRAFFIC_PER_UNIT else None),
                     "traffic_source": (ncu_traffic(res["build_kernel"], 1)[1]
                                        if res["build_kernel"] in NCU_TRAFFIC_PER_UNIT else
                                        "no capture of this kernel yet"),
                     "algorithmic_bytes": res["map_bytes"],
                     "timed": "the build call (this kernel alone), CUDA events on its stream",
                     "flop_per_launch": flop},
        "chain_roofline": {"bound": "hbm", "kernel": "affine_chain_ring_kernel<double>",
                           "achieved": res["map_bytes"] / comp_s / 1e9, "peak": peaks["hbm_gbs"],
                           "unit": "GB/s", "frac": res["map_bytes"] / comp_s / 1e9 / peaks["hbm_gbs"],
                           "algorithmic_bytes": res["map_bytes"]},
        "measured_alu_rates_tflops": {"fp64": fp64_rate / 1e12, "fp32": fp32_rate / 1e12},
        "gpu_launches": 2 * K,
        "clocks": res["clocks"],
        "variants": variants,
        "gpu_library_rates": peaks_probe,
        "peaks_file": peaks_src,
        "e2e": {"value": units / statistics.mean(e2e_t), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "api": "nv_build_propagators into maps allocated once + nv_compose, pinned host copies of "
                       "y0 and yT every step (host clock around each step)",
                "ms_per_step": statistics.mean(e2e_t) * 1e3,
                "nv_solve": {"value": units / statistics.mean(solve_t),
                             "ms_per_step": statistics.mean(solve_t) * 1e3,
                             "api": "nv_solve (allocates the 68.7 GB of maps, builds, composes, frees) + the "
                                    "same host copies"}},
    }
    if e2e_y is not None:
        line["e2e"]["bit_identical_to_device_run"] = bool(np.array_equal(e2e_y, res["yT"]))
        line["e2e"]["nv_solve"]["bit_identical_to_device_run"] = bool(np.array_equal(solve_y, res["yT"]))

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import nievergelt as nv
        cb = adv_cpu_baseline(w, m)
        (u1, t1, k1), (up, tp, kp) = cb["single"], cb["parallel"]
        t_ser = time.perf_counter()
        serial = nv.serial_fine(nv.workload_rhs(w, True), "rk4", w.t0, w.T, w.S, m, w.y0)
        t_ser = time.perf_counter() - t_ser
        line["cpu_baseline"] = {
            "value": up / tp, "unit": UNIT, "cores": cb["procs"], "kind": "oracle",
            "sample": f"FP64 numpy oracle map build of {kp} samples of {ADV_ORACLE_COLUMNS} basis columns "
                      f"(+ the solve from 0) of slices spread over the {w.S}, dealt over {cb['procs']} "
                      f"processes ({tp:.1f} s); one core: {k1} samples ({t1:.1f} s); the oracle's serial "
                      f"fine solve of the whole problem {t_ser:.1f} s",
            "single_core_value": u1 / t1}
        errs = {k: float(np.linalg.norm(v - serial) / np.linalg.norm(serial)) for k, v in results.items()}
        line["rel_err_vs_oracle"] = errs
        line["meets_target"] = {k: errs[k] <= ADV_TARGET[k.partition(":")[0]] for k in errs}
        line["target_note"] = ("relative L2 of the final state against the oracle's float64 serial fine "
                               "solve: 1e-11 float64, 1e-5 float32, 1e-4 refined reduced precision; plain "
                               "float32 maps sit above 1e-5 (the float32 rounding of the map entries "
                               "composes over 512 slices), one float64 pass brings them below it")
        fp64_err = errs["fp64"]
        eq = [k for k in errs if k != "fp64" and errs[k] <= max(fp64_err, 1e-11)]
        if eq:
            best = min(eq, key=lambda k: tts[k])
            line["time_to_solution_vs_plain_at_fixed_error"] = {
                "plain_fp64_ms": tts["fp64"], "best": best, "best_ms": tts[best],
                "speedup": tts["fp64"] / tts[best], "error_bound": max(fp64_err, 1e-11),
                "errors": {k: errs[k] for k in eq + ["fp64"]}}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def wave_flop_per_column_step(d):
    """Leapfrog on one basis column: the dense d x d product (d^2 FMA) and the
    update 2u - u_old + h^2 w (2 FMA per point), FMA = 2."""
    return 2 * d * (d + 2)


def run_wave(args):
    """Chebyshev spectral wave equation, M = 80 (d = 79, state 158), S = 512,
    T = 20, leapfrog dt = 8/M^2 (m = 32): float64 and float32 maps of the
    doubled state and their composition."""
    torch, world, rank, local = _device_setup()
    import numpy as np
    import paper_1304_6514_gb300 as nvp
    import workloads
    w = workloads.wave1d(S=args.slices, T=20.0 * args.slices / 512) if args.slices > 0 else workloads.wave1d()
    M = int(w.params[0])
    d = M - 1
    stream = torch.cuda.Stream()
    r = nvp.rhs("wave", w.dim, w.params)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    K, W = max(1, args.steps), max(3, args.warmup)
    out, clocks, m, h = {}, None, 0, 0.0
    fp64_rate = nvp.alu_rate("fp64", stream=stream)
    for prec in ("fp64", "fp32", "fp32_refine"):
        st = nvp.steps("leapfrog", w.dt, 0, prec)
        with torch.cuda.stream(stream):
            maps = nvp.build_propagators(r, w.t0, w.T, w.S, nvp.samples("affine"), st, stream=stream)
            info = nvp.maps_info(maps)
            m, h = info.steps_per_slice, info.h
            y0 = torch.tensor(workloads.wave1d_initial(M, h), device="cuda")
            yT = torch.empty_like(y0)
            for _ in range(W):
                nvp.build_propagators(r, w.t0, w.T, w.S, nvp.samples("affine"), st, maps=maps, stream=stream)
                nvp.compose(maps, y0, yT, stream=stream)
            ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
            sampler = ClockSampler(local) if prec == "fp64" else None
            stream.synchronize()
            if sampler:
                sampler.start()
            for k in range(K):
                flush.fill_(k & 0xFF)                       # maps fit in L2: flush before every step
                ev[k][0].record(stream)
                nvp.build_propagators(r, w.t0, w.T, w.S, nvp.samples("affine"), st, maps=maps, stream=stream)
                ev[k][1].record(stream)
                nvp.compose(maps, y0, yT, stream=stream)
                ev[k][2].record(stream)
            stream.synchronize()
            if sampler:
                clocks = sampler.stop()
            nvp.maps_check(maps, stream=stream)
        b = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
        c = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
        units = w.S * (w.dim + 1) * m
        out[prec] = {"build_ms": b, "compose_ms": c, "map_bytes": info.bytes,
                     "build_tflops": wave_flop_per_column_step(d) * units / (b * 1e-3) / 1e12,
                     "yT": yT.cpu().numpy()}
        maps.destroy()
    f64, f32, f32r = out["fp64"], out["fp32"], out["fp32_refine"]
    units = w.S * (w.dim + 1) * m
    step_ms = f64["build_ms"] + f64["compose_ms"]
    value, dev_s, _ = aggregate_over_ranks(units * K, step_ms * 1e-3 * K)
    for v in (f32, f32r):
        v["rel_err_vs_fp64_gpu"] = float(np.linalg.norm(v["yT"] - f64["yT"]) / np.linalg.norm(f64["yT"]))
    f32r["passes"] = 2
    results = {k: v["yT"] for k, v in out.items()}
    yT64 = f64["yT"]
    for v in out.values():
        v.pop("yT")
    flop = wave_flop_per_column_step(d) * units
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "M": M, "n": w.dim, "S": w.S, "steps_per_slice": m,
                       "l2": "flushed (256 MB write) before every timed step"},
            "variants": out, "time_to_solution_ms": {k: v["build_ms"] + v["compose_ms"] for k, v in out.items()},
            "roofline": {"bound": "alu", "kernel": "wave_build_kernel<double,80,2>",
                         "achieved": f64["build_tflops"], "peak": fp64_rate / 1e12, "unit": "TFLOP/s",
                         "frac": f64["build_tflops"] * 1e12 / fp64_rate,
                         "frac_of_nominal": f64["build_tflops"] * 1e12 / FP64_PEAK_NOMINAL,
                         "traffic": ncu_traffic("wave_build_kernel<double,80,2>", w.S * (w.dim + 1))[0]
                         if M == 80 else None,
                         "traffic_source": ncu_traffic("wave_build_kernel<double,80,2>", 1)[1],
                         "algorithmic_bytes": f64["map_bytes"],
                         "peak_source": "measured in this run: nv_alu_rate, FP64 FMA chains on every SM",
                         "flop_per_launch": flop},
            "gpu_launches": 3 * K, "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import wave as owave
        ns = min(w.S, 64)
        t0 = time.perf_counter()
        owave.build_affine(M, ns, m, h)
        el = time.perf_counter() - t0
        t0 = time.perf_counter()
        ys = owave.serial_fine(M, w.S, m, h, workloads.wave1d_initial(M, h))
        serial_s = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": ns * (w.dim + 1) * m / el, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"FP64 numpy oracle maps of {ns} of {w.S} slices ({el:.1f} s); "
                                          f"serial leapfrog solve {serial_s:.2f} s"}
        line["rel_err_vs_oracle_serial"] = {k: float(np.linalg.norm(v - ys) / np.linalg.norm(ys))
                                            for k, v in results.items()}
    if rank == 0:
        print(json.dumps(line))
    return 0


# The paper's GPU table (Section "graphics card implementation", Table gpuresults):
# y' = y^2 on [0, 1/2], (dt exponent, N slices, M nodes) and the printed time
# to solution in microseconds on a Tesla C2075 (backward Euler, Chebyshev
# interpolation, single precision, allocation and transfers included).
PAPER_GPU_TABLE = [(14, 32, 4, 193.6), (14, 64, 4, 187.5), (14, 128, 4, 208.4),
                   (15, 32, 5, 253.7), (15, 64, 5, 228.5), (15, 128, 5, 257.8),
                   (16, 32, 7, 388.3), (16, 64, 7, 338.9), (16, 128, 7, 392.0)]


def run_square(args):
    """The paper-shaped sweep of its GPU table: y' = y^2, y(0) = 1 on [0, 1/2],
    dt = 2^-14..2^-16, N = 32..128 slices, M = 4..7 nodes, float32 forward
    Euler with piecewise-linear tables on [0, 2].  Each configuration is timed
    end to end as the paper times it: nv_solve (allocate, build, compose, free)
    with the initial value copied from pinned host memory and the result copied
    back, plus the device time of build + compose on resident maps.  The line's
    value is the largest configuration's end-to-end throughput."""
    torch, world, rank, local = _device_setup()
    import numpy as np
    import paper_1304_6514_gb300 as nvp
    import workloads
    stream = torch.cuda.Stream()
    K, W = max(5, args.steps), max(3, args.warmup)
    r = nvp.rhs("square", 1)
    rows = []
    for e, S, M, paper_us in PAPER_GPU_TABLE:
        w = workloads.square_paper(e, S, M)
        smp = nvp.samples("pl1d", M, w.lo, w.hi)
        st = nvp.steps("euler", w.dt, 0, "fp32")
        hy0 = torch.tensor(w.y0, dtype=torch.float64).pin_memory()
        hyT = torch.empty(1, dtype=torch.float64).pin_memory()
        dy0 = torch.empty(1, dtype=torch.float64, device="cuda")
        dyT = torch.empty_like(dy0)
        with torch.cuda.stream(stream):
            def e2e():
                dy0.copy_(hy0, non_blocking=True)
                nvp.solve(r, w.t0, w.T, w.S, smp, st, dy0, dyT, stream=stream)
                hyT.copy_(dyT, non_blocking=True)
            for _ in range(W):
                e2e()
            stream.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
            for k in range(K):
                ev[k][0].record(stream)
                e2e()
                ev[k][1].record(stream)
            stream.synchronize()
            t_e2e = statistics.median(a.elapsed_time(b) for a, b in ev) * 1e3        # us
            maps = nvp.build_propagators(r, w.t0, w.T, w.S, smp, st, stream=stream)
            for _ in range(W):
                nvp.build_propagators(r, w.t0, w.T, w.S, smp, st, maps=maps, stream=stream)
                nvp.compose(maps, dy0, dyT, stream=stream)
            for k in range(K):
                ev[k][0].record(stream)
                nvp.build_propagators(r, w.t0, w.T, w.S, smp, st, maps=maps, stream=stream)
                nvp.compose(maps, dy0, dyT, stream=stream)
                ev[k][1].record(stream)
            stream.synchronize()
            t_dev = statistics.median(a.elapsed_time(b) for a, b in ev) * 1e3
            m = nvp.maps_info(maps).steps_per_slice
            maps.destroy()
            ys = torch.empty_like(dy0)
            nvp.serial_fine(r, w.t0, w.T, w.S, nvp.steps("euler", w.dt, 0, "fp64"), dy0, ys, stream=stream)
            stream.synchronize()
        exact = 1.0 / (1.0 - w.T)
        units = S * M * m
        rows.append({"dt": f"2^-{e}", "N": S, "M": M, "steps_per_slice": m, "e2e_us": t_e2e,
                     "device_us": t_dev, "traj_steps_per_s_e2e": units / (t_e2e * 1e-6),
                     "rel_err_method": abs(float(hyT[0]) - exact) / exact,
                     "rel_err_serial_fine_fp64": abs(float(ys[0]) - exact) / exact,
                     "paper_us_tesla_c2075": paper_us,
                     "paper_traj_steps_per_s": M * round(w.T / w.dt) / (paper_us * 1e-6)})
    big = rows[-1]
    # the paper's cost model (eq. gpucostmodel) fitted to these times, beside
    # its own fit on the Tesla C2075 (Table tauparameters)
    from paper_1304_6514_gb300 import costmodel
    shapes = [(0.5 * 2 ** e, S, M) for e, S, M, _ in PAPER_GPU_TABLE]
    fits = {}
    for key in ("e2e_us", "device_us"):
        tf, tn, tk = costmodel.fit_gpu_cost([(n, S, M, row[key]) for (n, S, M), row in zip(shapes, rows)])
        fits[key] = {"tau_F_us": tf, "tau_N_us": tn, "tau_K_us": tk}
    cost_model = {"model": "C_G = (M n / N) tau_F + N tau_N + tau_K, n = T / dt (eq. gpucostmodel)",
                  "fit_e2e": fits["e2e_us"], "fit_device": fits["device_us"],
                  "paper_tesla_c2075": {"tau_F_us": 0.040, "tau_N_us": 0.701, "tau_K_us": 137.0}}
    line = {"metric": METRIC, "value": big["traj_steps_per_s_e2e"], "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": big["e2e_us"] * 1e-3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 build, f64 composition", "data": "synthetic",
            "config": {"workload": "square_dt2^-16_N128_M7_euler_pl (paper GPU table shape)",
                       "l2": "not flushed: the whole problem (3.6 KB of tables) lives in L2 as in the paper's runs"},
            "e2e": {"value": big["traj_steps_per_s_e2e"], "unit": UNIT, "h2d_bytes_per_step": 8,
                    "d2h_bytes_per_step": 8, "api": "nv_solve (allocates, builds, composes, frees)"},
            "sweep": rows, "cost_model": cost_model,
            "paper_context": "Tesla C2075 (Fermi), backward Euler + Chebyshev interpolation, single precision; "
                             "times include allocation, transfers and CPU interpolation",
            "gpu_launches": 2 * K}
    if rank == 0:
        print(json.dumps(line))
    return 0


FP32_FLOP_PER_CHAIN_STEP = 220      # RK4 step of the 6-D chain incl. compensated update
MLP_FLOP_PER_SAMPLE_STEP = 6 * (7 * 256 + 2 * 256 * 256 + 256 * 6)   # fwd + bwd (2 + 4 x weights)


def _ev_ms(torch, fn, reps=1):
    fn()                                            # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def learned_equal_error(nvp, torch, np, w, r, net, count, train_ms):
    """Time to solution of `count` initial states at equal final-state error:
    the learned forms against the plain ones (all on this GPU, CUDA events)."""
    import workloads
    S = w.S
    st64, st32 = nvp.steps("rk4", w.dt), nvp.steps("rk4", w.dt, 0, "fp32")
    y0 = torch.tensor(workloads.Stream(21).uniform(count * 6, -0.5, 0.5).reshape(count, 6), device="cuda")
    fine = y0.clone()
    nvp.propagate(r, w.t0, w.T, S, st64, 0, S, fine)
    fine_h = fine.cpu().numpy()

    def err(y):
        y = y.cpu().numpy() if hasattr(y, "cpu") else y
        return float(np.max(np.linalg.norm(y - fine_h, axis=1) / np.linalg.norm(fine_h, axis=1)))

    yT = torch.empty_like(y0)
    errs = []
    for k in range(0, 10):
        net.parareal(r, w.t0, w.T, S, st64, k, y0, yT)
        torch.cuda.synchronize()
        errs.append(err(yT))
        if errs[-1] <= 1e-11:
            break
    y32 = y0.clone()
    nvp.propagate(r, w.t0, w.T, S, st32, 0, S, y32)
    e32 = err(y32)
    t64 = _ev_ms(torch, lambda: nvp.propagate(r, w.t0, w.T, S, st64, 0, S, y0.clone()))
    t32 = _ev_ms(torch, lambda: nvp.propagate(r, w.t0, w.T, S, st32, 0, S, y0.clone()))
    out = {"plain_f64_fine_ms": t64, "plain_f32_fine_ms": t32, "plain_f32_rel_err": e32,
           "parareal_rel_err_by_iteration": errs}
    k64 = next((k for k, e in enumerate(errs) if e <= 1e-11), None)
    if k64 is not None:
        # an NVTX range lets a profiler take exactly these launches (ncu --nvtx)
        torch.cuda.nvtx.range_push("learned_correction")
        tp = _ev_ms(torch, lambda: net.parareal(r, w.t0, w.T, S, st64, k64, y0, yT))
        torch.cuda.nvtx.range_pop()
        out["at_f64_error"] = {"error_bound": 1e-11, "parareal_iterations": k64, "parareal_ms": tp,
                               "plain_f64_ms": t64, "speedup_vs_plain": t64 / tp,
                               "amortised_parareal_ms": tp + train_ms}
    # the first iterations with float32 fine solves (nv_tune_set key 20), then float64 ones
    mixed = []
    for f32 in (2, 3):
        nvp.tune_set(20, f32)
        try:
            km = None
            for k in range(f32 + 1, 14):
                net.parareal(r, w.t0, w.T, S, st64, k, y0, yT)
                torch.cuda.synchronize()
                if err(yT) <= 1e-11:
                    km = k
                    break
            if km is not None:
                tm = _ev_ms(torch, lambda: net.parareal(r, w.t0, w.T, S, st64, km, y0, yT))
                mixed.append({"float32_iterations": f32, "iterations": km, "parareal_ms": tm,
                              "speedup_vs_plain": t64 / tm})
        finally:
            nvp.tune_set(20, 0)
    if mixed:
        best = dict(min(mixed, key=lambda x: x["parareal_ms"]))
        best["all"] = mixed
        out["at_f64_error_mixed"] = best
    k32 = next((k for k, e in enumerate(errs) if e <= e32), None)
    if k32 is not None:
        tp = _ev_ms(torch, lambda: net.parareal(r, w.t0, w.T, S, st64, k32, y0, yT))
        out["at_f32_error"] = {"error_bound": e32, "parareal_iterations": k32, "parareal_ms": tp,
                               "plain_f32_ms": t32, "speedup_vs_plain": t32 / tp}
    # the learned map alone, and plain RK4 with the coarsest step that reaches its error
    tl = _ev_ms(torch, lambda: net.compose(r, w.t0, w.T, S, st64, y0, yT))
    el = errs[0]
    coarse = None
    for mm in (1, 2, 4, 8, 16, 32, 64):
        yc = y0.clone()
        stc = nvp.steps("rk4", 0.0, mm, "fp32")
        nvp.propagate(r, w.t0, w.T, S, stc, 0, S, yc)
        ec = err(yc)
        if ec <= el:
            tc = _ev_ms(torch, lambda: nvp.propagate(r, w.t0, w.T, S, stc, 0, S, y0.clone()))
            coarse = {"steps_per_slice": mm, "dt": (w.T - w.t0) / S / mm, "ms": tc, "rel_err": ec}
            break
    out["at_learned_map_error"] = {"error_bound": el, "learned_compose_ms": tl,
                                   "plain_coarse_rk4_f32": coarse,
                                   "speedup_vs_plain": (coarse["ms"] / tl) if coarse else None}
    return out


def run_chain3_mlp(args):
    """Learned propagator for the 3-mass chain (S = 128, M = 65536 per slice):
    pair generation by the method's integrator (float32), MLP training on the
    tensor cores, validation against float64 end states, composition of 4096
    initial states through the learned map vs float64 fine integration."""
    torch, world, rank, local = _device_setup()
    import numpy as np
    import paper_1304_6514_gb300 as nvp
    import workloads
    w = workloads.chain3()
    S, M = w.S, w.per_dim
    r = nvp.rhs("chain3", 6)
    st32, st64 = nvp.steps("rk4", w.dt, 0, "fp32"), nvp.steps("rk4", w.dt)
    y0 = torch.empty(S * M * 6, dtype=torch.float32, device="cuda")
    ye = torch.empty_like(y0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    nvp.build_pairs(r, w.t0, w.T, S, st32, M, w.extra["seed"], -1.0, 1.0, y0, ye)   # warm-up
    ev[0].record()
    nvp.build_pairs(r, w.t0, w.T, S, st32, M, w.extra["seed"], -1.0, 1.0, y0, ye)
    ev[1].record()
    torch.cuda.synchronize()
    pairs_ms = ev[0].elapsed_time(ev[1])
    m = nvp.plan_steps(w.t0, w.T, S, w.dt)[0]
    pair_steps = S * M * m
    d = (ye - y0).view(-1, 6)[:65536].double().cpu().numpy()
    net = nvp.MLP(seed=1)
    net.set_scales([1 / np.sqrt(3)] * 6, list(d.std(axis=0)))
    sched = [(2000, 1e-3), (4000, 1e-3), (4000, 3e-4), (4000, 1e-4)]
    if args.train_steps > 0:
        sched = [(args.train_steps, 1e-3)]
    t0 = time.perf_counter()
    losses = [net.train(y0, ye, S, M, n, 4096, lr) for n, lr in sched]
    train_s = time.perf_counter() - t0
    nsteps = sum(n for n, _ in sched)
    Mv = 1024
    v0 = torch.empty(S * Mv * 6, dtype=torch.float64, device="cuda")
    ve = torch.empty_like(v0)
    nvp.build_pairs(r, w.t0, w.T, S, st64, Mv, w.extra["seed"] + 1, -1.0, 1.0, v0, ve)
    err = net.validate(v0, ve, S, Mv)
    fb = (err > 1e-3).astype(np.int32)
    equal_error = {str(c): learned_equal_error(nvp, torch, np, w, r, net, c, train_s * 1e3 + pairs_ms)
                   for c in [int(x) for x in args.learned_counts.split(",") if x]}
    train_tflops = MLP_FLOP_PER_SAMPLE_STEP * 4096 * nsteps / train_s / 1e12
    line = {"metric": METRIC, "value": pair_steps / (pairs_ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": 1, "warmup": 1, "ms_per_step": pairs_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 pairs, bf16 MLP (f32 accumulate), f64 reference", "data": "synthetic",
            "config": {"workload": w.name, "S": S, "M": M, "steps_per_slice": m, "hidden": [256, 256, 256],
                       "train_steps": nsteps, "batch": 4096},
            "pairs_ms": pairs_ms,
            "roofline": {"bound": "alu", "kernel": "pairs_kernel<float>",
                         "achieved": FP32_FLOP_PER_CHAIN_STEP * pair_steps / (pairs_ms * 1e-3) / 1e12,
                         "peak": FP32_PEAK_NOMINAL / 1e12, "unit": "TFLOP/s",
                         "frac": FP32_FLOP_PER_CHAIN_STEP * pair_steps / (pairs_ms * 1e-3) / FP32_PEAK_NOMINAL,
                         "traffic": ncu_traffic("pairs_kernel<float>", S * M * 12 * 4)[0],
                         "traffic_source": ncu_traffic("pairs_kernel<float>", 1)[1],
                         "algorithmic_bytes": S * M * 12 * 4},
            "train": {"seconds": train_s, "losses": losses, "model_tflops": train_tflops,
                      "steps_per_s": nsteps / train_s},
            "validation_rel_err": {"mean": float(err.mean()), "max": float(err.max()),
                                   "fallback_slices": int(fb.sum())},
            "equal_error": equal_error,
            "equal_error_note": ("time to solution of initial states at equal final-state error: the trained "
                                 "network as the coarse map of a float64 correction (k iterations: float64 "
                                 "defects of every slice, the correction chained over the network's 6 x 6 "
                                 "Jacobians at the learned composition; _mixed: the first 2 or 3 "
                                 "iterations with float32 fine solves) against the plain float64 / float32 fine integration of the same states, "
                                 "and the learned map alone against plain RK4 with the coarsest step that "
                                 "reaches its error; amortised = training + pair generation + the correction")}
    if rank == 0:
        print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.steps is None:
        args.steps = {"advdiff2d": 10, "heat1d": 100}.get(args.workload, 20)
    if args.variants is None:
        args.variants = ("fp32,fp32_refine,fp32_refine:2,bf16_refine" if args.workload == "advdiff2d"
                         else "fp32,tf32_refine,fp32_refine,fp32_refine:2")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "advdiff2d":
        return run_advdiff(args)
    if args.workload == "heat1d":
        return run_heat(args)
    if args.workload == "chain3_mlp":
        return run_chain3_mlp(args)
    if args.workload == "wave":
        return run_wave(args)
    if args.workload == "square":
        return run_square(args)
    if args.workload == "vdp_batch":
        return run_vdp_batch(args)
    if args.workload == "scalar":
        return run_scalar(args)
    raise SystemExit(f"unknown workload {args.workload}")


def run_heat(args):
    """--workload heat1d: u_t = u_xx + sin(pi x) cos t, n = 256, S = 1024, RK4
    m = 10, the float64 method as the line's value."""
    import numpy as np
    import torch

    world, rank, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1304_6514_gb300 import _build
    _build.build()                       # quiet: stdout carries only the JSON line
    import paper_1304_6514_gb300 as nvp
    import workloads

    w = workloads.heat1d(S=args.slices) if args.slices > 0 else workloads.heat1d()
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    K, W = args.steps, max(3, args.warmup)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- headline: float64 plain method
    sampler = ClockSampler(local)
    barrier()
    sampler.start()
    wall0 = time.perf_counter()
    res = time_variant(nvp, torch, w, "fp64", K, W, flush, stream)
    barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    m = res["m"]
    units = traj_steps(w, m)
    value, dev_s, _ = aggregate_over_ranks(units * K, sum(res["step_ms"]) * 1e-3)
    build_s = statistics.mean(res["build_ms"]) * 1e-3
    # the build reports the point-steps it integrated (the windowed builds count
    # only the rows each column's steps reach) and its kernel
    build_kernel = res["build_kernel"]
    horner_flop = FLOP_PER_COMPONENT_STEP * w.S * res["work_per_slice"]
    poly9 = "window" in build_kernel or "poly9" in build_kernel
    flop = (FLOP_PER_ROW_STEP_POLY9 if poly9 else FLOP_PER_COMPONENT_STEP) * w.S * res["work_per_slice"]
    rows = res["work_per_slice"] / ((w.dim + 1) * m)   # mean rows integrated per step and column
    flop_full = FLOP_PER_COMPONENT_STEP * units * w.dim
    achieved = flop / build_s
    fp64_rate = nvp.alu_rate("fp64", stream=stream)
    fp32_rate = nvp.alu_rate("fp32", stream=stream)

    # ---- variants
    variants = {"fp64": {"ms_per_step": statistics.mean(res["step_ms"]),
                         "build_ms": statistics.mean(res["build_ms"]),
                         "compose_ms": statistics.mean(res["compose_ms"]),
                         "traj_steps_per_s": units / (statistics.mean(res["step_ms"]) * 1e-3),
                         "build_tflops": achieved / 1e12,
                         "build_frac_of_measured_fp64": achieved / fp64_rate}}
    results = {"fp64": res["yT"]}
    for v in [x for x in args.variants.split(",") if x]:
        # "prec:p" sets p float64 correction passes (nv_tune_set key 5) for that variant
        prec, _, passes = v.partition(":")
        seq = None
        try:
            if passes:
                nvp.tune_set(5, int(passes))
            rv = time_variant(nvp, torch, w, prec, K, W, flush, stream)
            if prec == "fp32_refine":
                # the same passes one after another (tunable 10), for comparison
                nvp.tune_set(10, 1)
                seq = time_variant(nvp, torch, w, prec, K, W, flush, stream)
        except nvp.NvError as e:
            variants[v] = {"unavailable": str(e)}
            continue
        finally:
            if passes:
                nvp.tune_set(5, 0)
            nvp.tune_set(10, 0)
        results[v] = rv["yT"]
        bs = statistics.mean(rv["build_ms"]) * 1e-3
        variants[v] = {"ms_per_step": statistics.mean(rv["step_ms"]),
                       "build_ms": statistics.mean(rv["build_ms"]),
                       "compose_ms": statistics.mean(rv["compose_ms"]),
                       "traj_steps_per_s": units / (statistics.mean(rv["step_ms"]) * 1e-3),
                       "build_tflops": flop / bs / 1e12,
                       "build_frac_of_measured_fp32": flop / bs / fp32_rate,
                       "build_hbm_gbs": w.S * w.dim * (w.dim + 1) * (4 if prec != "fp64" else 8) / bs / 1e9,
                       "speedup_vs_fp64_plain": statistics.mean(res["step_ms"]) / statistics.mean(rv["step_ms"])}
        if seq is not None:
            variants[v]["sequential_passes"] = {
                "compose_ms": statistics.mean(seq["compose_ms"]),
                "bit_identical": bool(np.array_equal(seq["yT"], rv["yT"])),
                "note": "the default schedule runs the approximate chain, the defects and every "
                        "correction chain concurrently in one launch; this is the passes one after another"}
        ref = results["fp64"]
        variants[v]["rel_err_vs_fp64_gpu"] = float(np.linalg.norm(rv["yT"] - ref) / np.linalg.norm(ref))

    # ---- end to end through the one-call API with host buffers
    if args.no_e2e:
        e2e_t, h2d, d2h = [float("nan")], 0, 0
    else:
        e2e_t, h2d, d2h = time_e2e(nvp, torch, w, max(3, K // 4), 2, stream)
    e2e_val = units / statistics.mean(e2e_t)

    serial_ms, serial_gpu = time_serial_gpu(nvp, torch, w, stream)
    peaks_probe = {} if args.no_probe else gpu_peak_probe(torch)
    peaks, peaks_src = read_peaks()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": statistics.mean(res["step_ms"]), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(w, m, world),
        "time_to_solution_ms": statistics.mean(res["step_ms"]),
        "serial_fine_gpu": {"ms": serial_ms,
                            "rel_diff_method": float(np.linalg.norm(res["yT"] - serial_gpu) / np.linalg.norm(serial_gpu)),
                            "note": "one warp stepping all S m RK4 steps in sequence: the plain solve the "
                                    "method parallelises (the method does (d+1) times its work)"},
        "wall_s_timed_region": wall,
        "roofline": {"bound": "alu", "kernel": build_kernel,
                     "achieved": achieved / 1e12, "peak": fp64_rate / 1e12,
                     "unit": "TFLOP/s", "frac": achieved / fp64_rate,
                     "peak_source": "measured in this run: nv_alu_rate, FP64 FMA chains on every SM",
                     "frac_of_nominal": achieved / FP64_PEAK_NOMINAL,
                     "flop_per_unit": ("13 per row-step: the nine-point RK4 step the kernel executes "
                                       "(4 DADD + 1 DMUL + 4 DFMA)" if poly9 else
                                       "20 per row-step: the Horner-form RK4 step"),
                     "horner_unit_tflops": horner_flop / build_s / 1e12,
                     "rows_per_column": rows,
                     "rows_note": "each homogeneous column is integrated over windows holding the rows its "
                                  "steps reach (exactly zero elsewhere); the FLOPs count the rows integrated, "
                                  "rows_per_column is their mean over the m steps",
                     "full_width_equivalent_tflops": flop_full / build_s / 1e12,
                     "traffic": (ncu_traffic(build_kernel, w.S * w.dim)[0]
                                 if build_kernel in NCU_TRAFFIC_PER_UNIT else None),
                     "traffic_source": (ncu_traffic(build_kernel, 1)[1]
                                        if build_kernel in NCU_TRAFFIC_PER_UNIT else
                                        "no capture of this kernel yet"),
                     "algorithmic_bytes": w.S * w.dim * w.dim * 8,
                     "timed": "the build call (forcing-column kernel + this kernel, 97 % of it), CUDA events",
                     "flop_per_launch": flop},
        "gpu_launches": 3 * K,
        "clocks": clocks,
        "variants": variants,
        "gpu_library_rates": peaks_probe,
        "peaks_file": peaks_src,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "api": "nv_solve (allocates, builds, composes, frees) + pinned host copies",
                "ms_per_step": statistics.mean(e2e_t) * 1e3},
    }

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        done, el = oracle_sample(w, m)
        pdone, pel, procs = oracle_sample_parallel(w, m, el / done)
        serial, serial_s = oracle_serial(w, m)
        line["cpu_baseline"] = {
            "value": pdone * (w.dim + 1) * m / pel, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"FP64 numpy oracle map build of {pdone} of {w.S} slices over {procs} processes "
                      f"({pel:.1f} s); one core: {done} slices ({el:.1f} s); serial fine solve of the "
                      f"whole problem {serial_s:.2f} s",
            "single_core_value": done * (w.dim + 1) * m / el}
        line["rel_err_vs_oracle"] = {k: float(np.linalg.norm(v - serial) / np.linalg.norm(serial))
                                     for k, v in results.items()}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
