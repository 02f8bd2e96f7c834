"""Benchmark: limited element-stages per second of the kinetic-bounds limiter path.

One step = one SSP-RK3 time step of the whole path on the device (device time step,
then per stage: face traces, kinetic bounds, FR residual, stage update fused with the
limiter), i.e. 3 element-stages per element.  Default workload: the isentropic vortex
on a periodic 128 x 128 quad mesh, P3, 32 x 32 velocity grid, FP32-mixed bounds (the
FP64 path is timed beside it).  Inputs are resident in HBM; L2 (129 MB) is flushed
between timed steps because the state (8.4 MB) would otherwise stay cached.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload vortex|sedov|sod] [--precision fp32|fp64]

Multi-GPU runs (torchrun) are replicas: every rank runs the same workload and
`value` is the total over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "limited element-stages/sec (bounds+limit+RHS) on 1 GB300, FP32 vs FP64; % roofline"
UNIT = "element-stages/s"
SMS = 152
SM_MAX_MHZ = 2070.0
# The envelope loop of the FP32 bounds kernel needs, per (stencil state, velocity node),
# 2 products (g = Ex Ey and C g) and 4 comparisons (min and max of both): 6 FP32 lane-ops.
# Its roofline is the measured rate of exactly that instruction mix in a register-only loop
# (peaks/kbl_fp32_peaks.cu, `bench.py --peaks`): 155.5
# lane-ops per clock per SM (packed multiplies and three-input min/max issue to two pipes
# that overlap only in part), times 152 SMs and the 2070 MHz maximum clock.
OPS_PER_STATE_NODE = 6.0
LANE_OPS_PER_CLK_SM = 155.5
PEAK_SOURCE = ("measured envelope-pattern rate 155.5 FP32 lane-ops/clk/SM (bench.py --peaks) "
               "x 152 SMs x 2070 MHz")
# DRAM bytes (read + write) of one launch of the FP32 2D bounds kernel on the vortex workload,
# from an ncu capture of that kernel (dram__bytes_read.sum + dram__bytes_write.sum).  Must be
# reset to None whenever that kernel changes, until it is captured again.
BOUNDS_F32_VORTEX_TRAFFIC = 17076992


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="vortex",
                    choices=["vortex", "sedov", "sod", "batched", "adjoint", "triangles"])
    ap.add_argument("--adj-n", type=int, default=256, help="adjoint workload: elements per axis")
    ap.add_argument("--adj-steps", type=int, default=100, help="adjoint workload: time steps per gradient")
    ap.add_argument("--adj-cfl", type=float, default=0.05, help="adjoint workload: CFL number")
    ap.add_argument("--peaks", action="store_true",
                    help="build and run the FP32 instruction-rate microbenchmark behind the roofline peak")
    ap.add_argument("--batch-problems", type=int, default=4096)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-fp64-leg", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-subworkloads", action="store_true",
                    help="vortex only: skip the Sedov and batched sub-objects of the default line")
    ap.add_argument("--bounds-tile", type=int, default=-1, help="FP32 bounds thread tile (0: 4x4, 1: 4x2, 2: 2x4; -1: default)")
    ap.add_argument("--rhs-overlap", type=int, default=1, choices=[0, 1],
                    help="1: each stage's residual on a graph branch beside its bounds (default); 0: serial")
    ap.add_argument("--rhs-tc", action="store_true",
                    help="FP32-mixed residual of P2/P3 on the tensor cores (off by default: slower, see the header)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def workload(name):
    """2D cases step at CFL 0.05: with dt = cfl * min over axes of h / (|u| + c), SSP-RK3 with
    P2-P3 flux reconstruction is linearly stable below about half the 1D limit 1 / (2p + 1)."""
    from paper_2407_20966_gb300 import inputs
    if name == "vortex":
        mesh, ic = inputs.isentropic_vortex(128)
        return dict(name="isentropic vortex 128x128 P3, 32x32 velocity grid, periodic",
                    dim=2, p=3, nu=(32, 32), mesh=mesh, ic=ic, cfl=0.05)
    if name == "sedov":
        mesh, ic = inputs.sedov(512)
        # HLL: the Riemann solver of the paper's own Sedov run (Sec. 6.6)
        return dict(name="Sedov blast 512x512 P2, 32x32 velocity grid, HLL flux", dim=2, p=2, nu=(32, 32),
                    mesh=mesh, ic=ic, cfl=0.05, flux=2)
    mesh, ic = inputs.sod(200)
    # the stencil this configuration names: own nodes and both face-neighbour elements' nodes
    return dict(name="Sod shock tube 200 P3, 64 velocity points, stencil of own and both neighbours' nodes",
                dim=1, p=3, nu=(64,), mesh=mesh, ic=ic, cfl=0.1, stencil=1)


def stencil_size(wl):
    n = wl["p"] + 1
    ns = n ** wl["dim"]
    nfp = 2 if wl["dim"] == 1 else 4 * n
    return 3 * ns if wl.get("stencil", 0) == 1 else ns + 2 * nfp


def nu_total(wl):
    return int(np.prod(wl["nu"]))


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != 6:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[2:]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        sm = sorted(r[0] for r in rows)
        loaded = [s for s in sm if s > 0.5 * rows[0][1]] or sm
        return {"sm_mhz": float(np.median(loaded)), "sm_max_mhz": rows[0][1], "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# replicas: the slowest rank's time defines the job's time
# ---------------------------------------------------------------------------
def max_over_ranks(ms, device=None):
    """Max of a per-rank time over the process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier_world():
    """Barrier over the process group (if any) and its size."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()
        return dist.get_world_size()
    return 1


def job_throughput(units_per_rank, ms_max, world):
    """Whole-job units per second: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (ms_max * 1e-3)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world):
    import torch
    from paper_2407_20966_gb300 import build, inputs, kbl

    build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wl = workload(args.workload)
    precision = kbl.FP32_MIXED if args.precision == "fp32" else kbl.FP64
    mesh = wl["mesh"]
    E = mesh.n_elem

    def make_ctx(prec):
        ctx = kbl.Context(dim=wl["dim"], p=wl["p"], nu=wl["nu"], precision=prec, flux=wl.get("flux", 0),
                          stencil=wl.get("stencil", 0))
        ctx.mesh_upload(mesh.nbr, mesh.h, mesh.bc)
        return ctx

    ctx = make_ctx(precision)
    if args.bounds_tile >= 0:
        ctx.set_tuning(kbl.TUNE_BOUNDS_TILE, args.bounds_tile)
    if args.rhs_tc:
        ctx.set_tuning(kbl.TUNE_RHS_TC, 1)
    if not args.rhs_overlap:
        ctx.set_tuning(kbl.TUNE_RHS_OVERLAP, 0)
    xi = ctx.operator(kbl.OP_NODES)
    w0 = inputs.nodal_field(mesh, xi, wl["ic"])
    w_dev = torch.from_numpy(w0).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def timed_steps(c, w, K, W):
        c.set_time(0.0)
        for _ in range(W):
            c.step(w, wl["cfl"])
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        l0 = c.launch_count()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for k in range(K):
            flush.zero_()
            evs[k][0].record(stream)
            c.step(w, wl["cfl"])
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        c.check()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        return ms, c.launch_count() - l0

    with ClockSampler(dev.index) as clk:
        ms, launches = timed_steps(ctx, w_dev, args.steps, args.warmup)
    clocks = clk.summary()
    ms = max_over_ranks(ms, dev)
    value = job_throughput(E * 3 * args.steps, ms, world)

    # dominant kernel: the bounds kernel, timed per launch with events on the launching
    # stream, same workload and launch configuration as inside the step
    wf = torch.zeros((ctx.nv, E, ctx.nfp), dtype=torch.float64, device=dev)
    bnd = torch.zeros((2, ctx.nv, E), dtype=torch.float64, device=dev)
    w_dev.copy_(torch.from_numpy(w0))
    ctx.traces(w_dev, wf)
    for _ in range(3):
        ctx.bounds(w_dev, wf, bnd)
    kb = max(10, args.steps)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(kb)]
    for k in range(kb):
        flush.zero_()
        evs[k][0].record(stream)
        ctx.bounds(w_dev, wf, bnd)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    bounds_ms = sum(a.elapsed_time(b) for a, b in evs) / kb
    nS, NU = stencil_size(wl), nu_total(wl)
    ops_per_launch = OPS_PER_STATE_NODE * nS * NU * E   # 2 products + 4 comparisons per (state, node)
    achieved = ops_per_launch / (bounds_ms * 1e-3) / 1e12
    peak = LANE_OPS_PER_CLK_SM * SMS * SM_MAX_MHZ * 1e6 / 1e12
    traffic = BOUNDS_F32_VORTEX_TRAFFIC if (args.workload == "vortex" and precision == kbl.FP32_MIXED
                                             and args.bounds_tile <= 0) else None
    roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "T FP32 lane-ops/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": "k_bounds2d_f32" if (
                    wl["dim"] == 2 and precision == kbl.FP32_MIXED) else "bounds",
                "bounds_ms_per_launch": round(bounds_ms, 4), "work": "6 lane-ops per (stencil state, velocity node)",
                "peak_source": PEAK_SOURCE}

    # FP64 leg (same workload, FP64 bounds)
    fp64 = None
    if not args.no_fp64_leg and precision != kbl.FP64:
        c64 = make_ctx(kbl.FP64)
        w64 = torch.from_numpy(w0).to(dev)
        k64 = max(3, min(args.steps, 10))
        ms64, _ = timed_steps(c64, w64, k64, 1)
        fp64 = {"value": E * 3 * k64 / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64 / k64}
        c64.close()

    # end to end through the C-ABI with host buffers (pinned): an ensemble of independent states
    # of the workload (the initial state with a seeded 1e-6 perturbation per member), one step
    # each; every member pays its H2D copy and the D2H copy of its result, which
    # kbl_run_host_ensemble overlaps with the neighbouring members' steps
    M = 16
    rng = np.random.default_rng(1)
    ens = np.ascontiguousarray(np.stack([w0 * (1 + 1e-6 * rng.uniform(-1, 1, w0.shape)) for _ in range(M)]))
    w_pin = torch.from_numpy(ens).pin_memory()
    out_pin = torch.empty_like(w_pin).pin_memory()
    win, wout = w_pin.numpy(), out_pin.numpy()
    ctx.set_time(0.0)
    ctx.run_host_ensemble(win, wout, 1, wl["cfl"])
    ke = max(3, min(args.steps // 4, 8))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        ctx.run_host_ensemble(win, wout, 1, wl["cfl"])
    e2e_s = (time.perf_counter() - t0) / (ke * M)
    nbytes = w0.nbytes
    e2e = {"value": E * 3 / e2e_s * world, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes, "call": f"kbl_run_host_ensemble, {M} members x 1 step, pinned host buffers"}
    ctx.set_time(0.0)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if precision == kbl.FP32_MIXED else "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "elements": E, "stages_per_step": 3,
                       "precision": args.precision, "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": f"replicas x{world}"},
            "fp64": fp64, "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "clocks": clocks}
    return line, w0, wl


# ---------------------------------------------------------------------------
# CPU checker timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def _oracle_block(wl):
    """The bounded CPU sample of a workload: a 16 x 16 block of elements of the 2D mesh
    (periodic within the block), or the whole 1D mesh."""
    import oracle as orc
    from paper_2407_20966_gb300 import inputs
    cfg = orc.Config(dim=wl["dim"], p=wl["p"], nu=tuple(wl["nu"]), flux=wl.get("flux", 0),
                     stencil=wl.get("stencil", 0))
    xi, _ = orc.gauss_legendre(wl["p"] + 1)
    mesh = wl["mesh"]
    if wl["dim"] == 2:
        nx = mesh.n[0]
        b = 16
        i0 = max(0, nx // 2 - b // 2)
        sub = inputs.mesh_2d(b, b, 0.0, 1.0, 0.0, 1.0, periodic=(True, True))
        ids = np.array([(i0 + iy) * nx + (i0 + ix) for iy in range(b) for ix in range(b)])
        w = inputs.nodal_field(mesh, xi, wl["ic"])[:, ids, :]
        om = orc.Mesh(sub.nbr, mesh.h[ids], mesh.bc)
        desc = f"{b}x{b} element block of the workload, periodic within the block"
    else:
        w = inputs.nodal_field(mesh, xi, wl["ic"])
        om = orc.Mesh(mesh.nbr, mesh.h, mesh.bc)
        desc = "whole mesh"
    return cfg, om, np.ascontiguousarray(w), desc


def _oracle_steps(wl_name, budget_s, max_steps=200):
    """Run the checker's SSP-RK3 steps on the bounded sample until the budget is spent; returns
    (element-stages, seconds, steps, description).  Also the body of each parallel worker."""
    import oracle as orc
    wl = workload(wl_name)
    cfg, om, w, desc = _oracle_block(wl)
    dt = orc.dt(cfg, om, w, wl["cfl"])
    n, t0 = 0, time.perf_counter()
    while True:
        w, _ = orc.ssprk3_step(cfg, om, w, dt)
        n += 1
        el = time.perf_counter() - t0
        if el > budget_s or n >= max_steps:
            break
    return om.n_elem * 3 * n, el, n, f"{desc} ({om.n_elem} elements)"


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(wl_name, budget_s=12.0, workers=None):
    """Time the FP64 CPU checker, as it stands, on a bounded sample of the workload: one process
    on one core, then (workers > 1) one independent replica of the same sample per host core in a
    spawn-started process pool, the total over the wall time of the slowest."""
    import oracle as orc
    orc.build()
    units, el, n, desc = _oracle_steps(wl_name, budget_s)
    single = {"value": units / el, "unit": UNIT, "cores": 1, "kind": "oracle",
              "sample": f"{n} SSP-RK3 steps on a {desc}, {el:.1f} s"}
    workers = host_cores() if workers is None else workers
    if workers <= 1:
        return single
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(workers) as pool:
        res = pool.starmap(_oracle_steps, [(wl_name, budget_s, 10 ** 9)] * workers)
    wall = time.perf_counter() - t0
    total = sum(r[0] for r in res)
    slowest = max(r[1] for r in res)
    return {"value": total / slowest, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"{workers} independent replicas (one per host core, spawn pool), each "
                      f"{res[0][2]}+ SSP-RK3 steps on a {desc} for {budget_s:.0f} s; {wall:.1f} s wall",
            "single_core": single}


def oracle_batch_sample(probs, budget_s=12.0):
    """The FP64 CPU checker on the first problems of the batch (whole problems, one core)."""
    import oracle as orc
    from paper_2407_20966_gb300 import inputs
    orc.build()
    n_el, steps, t0 = 0, 0, time.perf_counter()
    done = []
    for p, m, ic in probs:
        cfg = orc.Config(dim=2, p=p, nu=(32, 32))
        om = orc.Mesh(m.nbr, m.h, m.bc)
        xi, _ = orc.gauss_legendre(p + 1)
        w = inputs.nodal_field(m, xi, ic)
        w, _ = orc.ssprk3_step(cfg, om, w, orc.dt(cfg, om, w, 0.05))
        n_el += m.n_elem
        steps += 1
        done.append(f"{m.n[0]}x{m.n[1]} P{p}")
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": n_el * 3 / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one SSP-RK3 step of the first {steps} batch problems ({', '.join(done)}), {el:.1f} s"}


def run_reference(args, rank):
    budget = max(5.0, min(60.0, 4.0 * (args.steps + args.warmup)))
    if args.workload == "adjoint":
        return {"impl": "reference", "unavailable": "the FP64 CPU oracle has no reverse mode (forward only)"}
    if args.workload == "batched":
        from paper_2407_20966_gb300 import inputs
        probs = inputs.four_quadrant_batch(0x5EED, args.batch_problems)
        cb = oracle_batch_sample(probs, budget_s=budget)
        wl = {"name": f"batched: {args.batch_problems} four-quadrant Riemann problems (CPU sample)"}
    else:
        wl = workload(args.workload)
        cb = oracle_sample(args.workload, budget_s=0.5 * budget)
    return {"metric": METRIC, "value": cb["value"], "unit": UNIT, "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl["name"]}, "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def batch_stencil_nodes(b):
    """Sum over the batch's elements of |S| N_u: the (stencil state, velocity node) pairs of one
    bounds launch, |S| = (p+1)^2 + 8 (p+1), N_u = 32 x 32."""
    n = b.p.astype(np.int64) + 1
    return int(((n * n + 8 * n) * b.n_elem.astype(np.int64)).sum() * 32 * 32)


def run_batched(args, rank, world, steps=None, warmup=None):
    """The batched form: 4096 independent four-quadrant problems (seed 0x5EED), n x n elements with
    n ~ U{16..128}, orders P1..P4, 32 x 32 velocity grid, FP32-mixed, one persistent launch per
    phase, one graph per step, launch shape from the autotuner.  The roofline is taken on a
    bounds launch over the whole batch in the tuned shape (CUDA events on the batch's stream);
    the e2e figure goes through kbl_batch_run_host (groups of problems whose copies overlap)."""
    import torch
    from paper_2407_20966_gb300 import build, inputs, kbl

    build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    K = args.steps if steps is None else steps
    W = args.warmup if warmup is None else warmup
    probs = inputs.four_quadrant_batch(0x5EED, args.batch_problems)
    b = kbl.Batch([(p, m.nbr, m.h, m.bc) for p, m, _ in probs])
    E = int(b.elem_offsets[-1])
    w0 = inputs.batch_state(probs, b.nodes, b.state_offsets)
    wd = torch.from_numpy(w0).to(dev)
    b.autotune(wd)
    cfl = 0.05   # below the DG / SSP-RK3 limit of about 1 / (2p + 1) for every order in the batch
    for _ in range(max(1, W)):
        b.step(wd, cfl)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    stream = torch.cuda.current_stream()
    l0 = b.launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with ClockSampler(dev.index) as clk:
        for k in range(K):
            evs[k][0].record(stream)
            b.step(wd, cfl)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    b.check()
    launches = b.launch_count() - l0
    ms = max_over_ranks(sum(a.elapsed_time(c) for a, c in evs), dev)
    value = job_throughput(E * 3 * K, ms, world)
    # the same steps as ONE persistent launch per step (the other form), for comparison
    b.set_form(1)
    b.step(wd, cfl)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kp = 2
    e0.record(stream)
    for _ in range(kp):
        b.step(wd, cfl)
    e1.record(stream)
    torch.cuda.synchronize()
    b.check()
    one_launch_ms = e0.elapsed_time(e1) / kp
    b.set_form(0)
    # dominant kernel: the bounds phase over the whole batch, tuned shape, timed alone
    bnd = torch.zeros(8 * E, dtype=torch.float64, device=dev)
    b.bounds(wd, bnd)
    bms = []
    for _ in range(3):
        b.bounds(wd, bnd)
        bms.append(b.bounds_ms())
    bounds_ms = float(np.mean(bms))
    peak = LANE_OPS_PER_CLK_SM * SMS * SM_MAX_MHZ * 1e6 / 1e12
    achieved = OPS_PER_STATE_NODE * batch_stencil_nodes(b) / (bounds_ms * 1e-3) / 1e12
    del bnd
    # end to end: the whole batch from pinned host memory, one step, back to pinned host memory
    w_pin = torch.from_numpy(w0).pin_memory()
    out_pin = torch.empty_like(w_pin).pin_memory()
    b.run_host(w_pin.numpy(), out_pin.numpy(), 1, cfl)
    ke = 2
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        b.run_host(w_pin.numpy(), out_pin.numpy(), 1, cfl)
    e2e_s = (time.perf_counter() - t0) / ke
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"batched: {b.P} four-quadrant Riemann problems, n x n elements n~U[16,128], "
                                   f"P1..P4, 32x32 velocity grid, FP32-mixed, persistent launches + graph",
                       "elements": E, "problems": b.P, "stages_per_step": 3, "tuning": b.tuning(),
                       "l2": "state (%.1f GB) larger than L2" % (w0.nbytes / 1e9),
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": E * 3 * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": w0.nbytes,
                    "d2h_bytes_per_step": w0.nbytes,
                    "call": "kbl_batch_run_host, 1 step, pinned host buffers, copies overlapped by problem groups"},
            "gpu_launches": launches,
            "form": {"timed": "one persistent launch per phase, 14 per step, in one graph",
                     "one_launch_ms_per_step": one_launch_ms,
                     "one_launch": "the whole step as one persistent launch with per-problem dataflow"},
            "roofline": {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3),
                         "unit": "T FP32 lane-ops/s", "frac": round(achieved / peak, 4), "traffic": None,
                         "kernel": "k_batch_bounds", "bounds_ms_per_launch": round(bounds_ms, 3),
                         "work": "6 lane-ops per (stencil state, velocity node)",
                         "measured_on": "one bounds launch over the whole batch in the tuned launch shape",
                         "peak_source": PEAK_SOURCE},
            "clocks": clk.summary()}
    b.close()
    del wd, w_pin, out_pin
    torch.cuda.empty_cache()
    return line, probs, b


def run_sub_mesh(args, name, steps, warmup, dev):
    """A second single-mesh workload timed like the headline (L2 flushed between steps, CUDA
    events on the launching stream), with its own clock record and bounds roofline; FP64 beside."""
    import torch
    from paper_2407_20966_gb300 import inputs, kbl
    wl = workload(name)
    mesh = wl["mesh"]
    E = mesh.n_elem
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def make_ctx(prec):
        c = kbl.Context(dim=wl["dim"], p=wl["p"], nu=wl["nu"], precision=prec, flux=wl.get("flux", 0),
                        stencil=wl.get("stencil", 0))
        c.mesh_upload(mesh.nbr, mesh.h, mesh.bc)
        return c

    def timed(c, w, K, W):
        c.set_time(0.0)
        for _ in range(W):
            c.step(w, wl["cfl"])
        torch.cuda.synchronize()
        _barrier_world()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for k in range(K):
            flush.zero_()
            evs[k][0].record(stream)
            c.step(w, wl["cfl"])
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        c.check()
        return max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), dev)

    ctx = make_ctx(kbl.FP32_MIXED)
    w0 = inputs.nodal_field(mesh, ctx.operator(kbl.OP_NODES), wl["ic"])
    wd = torch.from_numpy(w0).to(dev)
    with ClockSampler(dev.index) as clk:
        ms = timed(ctx, wd, steps, warmup)
    wd.copy_(torch.from_numpy(w0))
    wf = torch.zeros((ctx.nv, E, ctx.nfp), dtype=torch.float64, device=dev)
    bnd = torch.zeros((2, ctx.nv, E), dtype=torch.float64, device=dev)
    ctx.traces(wd, wf)
    for _ in range(2):
        ctx.bounds(wd, wf, bnd)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a, z in evs:
        flush.zero_()
        a.record(stream)
        ctx.bounds(wd, wf, bnd)
        z.record(stream)
    torch.cuda.synchronize()
    bounds_ms = sum(a.elapsed_time(z) for a, z in evs) / len(evs)
    achieved = OPS_PER_STATE_NODE * stencil_size(wl) * nu_total(wl) * E / (bounds_ms * 1e-3) / 1e12
    peak = LANE_OPS_PER_CLK_SM * SMS * SM_MAX_MHZ * 1e6 / 1e12
    ctx.close()
    c64 = make_ctx(kbl.FP64)
    k64 = 2
    ms64 = timed(c64, torch.from_numpy(w0).to(dev), k64, 1)
    c64.close()
    world = _barrier_world()
    return {"workload": wl["name"], "elements": E, "value": job_throughput(E * 3 * steps, ms, world), "unit": UNIT,
            "ms_per_step": ms / steps, "steps": steps, "warmup": warmup, "precision": "fp32",
            "l2": "flushed between timed steps (256 MB write)",
            "fp64": {"value": job_throughput(E * 3 * k64, ms64, world), "unit": UNIT, "ms_per_step": ms64 / k64},
            "roofline": {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3),
                         "unit": "T FP32 lane-ops/s", "frac": round(achieved / peak, 4), "traffic": None,
                         "kernel": "k_bounds2d_f32", "bounds_ms_per_launch": round(bounds_ms, 4),
                         "work": "6 lane-ops per (stencil state, velocity node)", "peak_source": PEAK_SOURCE},
            "clocks": clk.summary()}


def run_triangles(args, steps, warmup, dev):
    """Affine triangles (Sec. 5: Williams-Shunn P2 solution points, 3 Gauss-Legendre points per
    edge): 2 x 256 x 256 jittered periodic triangles on [0,1]^2, 32 x 32 velocity grid, FP32-mixed
    bounds and residual, FP64 traces and limiter, HLLC, fixed dt at CFL 0.05.  One step is
    kbl_tri_step: per stage the bounds of the 24-state stencils (gathered in the kernel), the
    residual beside them, the combination with the traces of its result, the node-set limiter.  Timed like the headline (L2 flushed between steps); the roofline is the
    step's bounds launch (kbl_tri_bounds) over the whole mesh, timed alone with CUDA events."""
    import numpy as np
    import torch
    from paper_2407_20966_gb300 import inputs, kbl
    m = inputs.tri_mesh_2d(256, 256, 0.0, 1.0, 0.0, 1.0, jitter=0.2, seed=17)
    E = m.n_elem
    tm = kbl.TriMesh(2, m.xy, m.nbr, m.nbr_edge, m.bc, precision=kbl.FP32_MIXED, flux=1, nu=(32, 32))
    rs, _ = kbl.tri_points(2)
    w0 = inputs.tri_nodal_field(m, rs, inputs.tri_blast)
    wd = torch.from_numpy(w0).to(dev)
    dt = tm.dt(wd, 0.05)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        tm.step(wd, dt)
    torch.cuda.synchronize()
    world = _barrier_world()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with ClockSampler(dev.index) as clk:
        for k in range(steps):
            flush.zero_()
            evs[k][0].record(stream)
            tm.step(wd, dt)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    tm.check()
    ms = max_over_ranks(sum(a.elapsed_time(z) for a, z in evs), dev)
    # dominant kernel: the step's bounds launch (stencils gathered in the kernel) over the whole mesh
    wf = torch.zeros(E, tm.nfp, 4, dtype=torch.float64, device=dev)
    bnd = torch.zeros(2, 4, E, dtype=torch.float64, device=dev)
    tm.traces(wd, wf)
    tm.bounds(wd, wf, bnd)
    bev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a, z in bev:
        flush.zero_()
        a.record(stream)
        tm.bounds(wd, wf, bnd)
        z.record(stream)
    torch.cuda.synchronize()
    tm.check()
    bounds_ms = sum(a.elapsed_time(z) for a, z in bev) / len(bev)
    achieved = OPS_PER_STATE_NODE * tm.nstencil * 32 * 32 * E / (bounds_ms * 1e-3) / 1e12
    peak = LANE_OPS_PER_CLK_SM * SMS * SM_MAX_MHZ * 1e6 / 1e12
    # end to end: pinned host state in, one step, pinned host state out
    w_pin = torch.from_numpy(w0).pin_memory()
    out_pin = torch.empty_like(w_pin).pin_memory()
    ke = 3
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        wd.copy_(w_pin, non_blocking=True)
        tm.step(wd, dt)
        out_pin.copy_(wd, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / ke
    tm.close()
    return {"workload": f"triangles: {E} periodic jittered P2 triangles (Williams-Shunn points), 32x32 velocity "
                        f"grid, FP32-mixed bounds, HLLC, smoothed blast", "elements": E,
            "value": job_throughput(E * 3 * steps, ms, world), "unit": UNIT, "ms_per_step": ms / steps,
            "steps": steps, "warmup": warmup, "l2": "flushed between timed steps (256 MB write)",
            "e2e": {"value": job_throughput(E * 3, max_over_ranks(e2e_s * 1e3, dev), world), "unit": UNIT,
                    "h2d_bytes_per_step": int(w0.nbytes),
                    "d2h_bytes_per_step": int(w0.nbytes),
                    "call": "pinned host copy in, kbl_tri_step, pinned host copy out"},
            "roofline": {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3),
                         "unit": "T FP32 lane-ops/s", "frac": round(achieved / peak, 4), "traffic": None,
                         "kernel": "k_bounds_tri_f32", "bounds_ms_per_launch": round(bounds_ms, 4),
                         "work": "6 lane-ops per (stencil state, velocity node), 24 states per element",
                         "peak_source": PEAK_SOURCE},
            "clocks": clk.summary()}


def run_adjoint(args, rank, world):
    """Reverse mode: the gradient of the integrated entropy at t_end with respect to the initial
    state of the shock-vortex problem (n x n P3, 32 x 32 velocity grid, FP64, CFL 0.05) through
    `adj_steps` limited SSP-RK3 steps, checkpoints every 10 steps.  One timed unit is one whole
    gradient: the checkpointed forward pass plus the backward pass (segment recomputation and
    the adjoint kernels).  Warm-up: gradients of 2-step trajectories.  `value` counts the forward
    element-stages differentiated per second of that whole computation."""
    import torch
    from paper_2407_20966_gb300 import adjoint, build, inputs, kbl

    build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    n, n_steps, every, cfl = args.adj_n, args.adj_steps, 10, args.adj_cfl
    mesh, ic = inputs.shock_vortex(n)
    ctx = kbl.Context(dim=2, p=3, nu=(32, 32), precision=kbl.FP64, eps_rule=1)
    ctx.mesh_upload(mesh.nbr, mesh.h, mesh.bc)
    w0 = inputs.nodal_field(mesh, ctx.operator(kbl.OP_NODES), ic)
    E = mesh.n_elem
    wd0 = torch.from_numpy(w0).to(dev)
    dts = adjoint.cfl_time_steps(ctx, wd0, n_steps, cfl)
    ctx.counters()
    w = wd0.clone()
    for dt in dts:
        ctx.step_fixed(w, dt)
    st, cnt = ctx.counters()

    def gradient(steps):
        x = wd0.clone().requires_grad_(True)
        J = adjoint.entropy(adjoint.trajectory(x, ctx, steps, checkpoint_every=every), ctx)
        J.backward()
        return J.detach(), x.grad

    for _ in range(max(1, args.warmup)):
        gradient(dts[:2])
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    K = max(1, args.steps)
    l0 = ctx.launch_count()
    times = []
    with ClockSampler(dev.index) as clk:
        for _ in range(K):
            a, m, b = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(stream)
            x = wd0.clone().requires_grad_(True)
            y = adjoint.trajectory(x, ctx, dts, checkpoint_every=every)
            J = adjoint.entropy(y, ctx)
            m.record(stream)
            J.backward()
            b.record(stream)
            torch.cuda.synchronize()
            times.append((a.elapsed_time(m), m.elapsed_time(b)))
    ctx.check()
    launches = ctx.launch_count() - l0
    g = x.grad
    ms = max_over_ranks(sum(f + r for f, r in times), dev)
    value = job_throughput(E * 3 * n_steps * K, ms, world)
    fwd = sum(f for f, _ in times) / K
    bwd = sum(r for _, r in times) / K
    line = {"metric": METRIC, "value": value, "unit": "differentiated element-stages/s", "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"adjoint: shock-vortex on [0,2]x[0,1], {n}x{n} P3 (Mach 1.1 stationary shock, isentropic "
                                   f"vortex), 32x32 velocity grid, FP64, CFL {cfl}, gradient of the integrated "
                                   f"entropy through {n_steps} limited SSP-RK3 steps, checkpoints every {every}",
                       "elements": E, "time_steps": n_steps, "t_end": float(sum(dts)),
                       "limited_element_stages": int(cnt["limited_elements"]),
                       "forward_ms": fwd, "backward_ms": bwd, "J": float(J.item()),
                       "grad_max_abs": float(g.abs().max().item()),
                       "l2": "state (%.1f MB) x checkpoints; steps stream through more than L2" % (w0.nbytes / 1e6),
                       "parallelism": f"replicas x{world}"},
            "gpu_launches": launches,
            "clocks": clk.summary()}
    return line, w0, workload("vortex")


def run_peaks():
    """Compile and run the register-only rate probes under peaks/ (measurement code beside this
    file, not part of the library):
    FP32 multiply and min/max rates, alone and in the envelope pattern (kbl_fp32_peaks.cu),
    then the integer and FP64 operations the other kernels spend (kbl_int_fp64_rates.cu), per
    SM clock (clock64 inside each block); clocks sampled beside."""
    import subprocess
    here = os.path.dirname(os.path.abspath(__file__))
    out_dir = os.path.join(here, "paper_2407_20966_gb300", "_build")
    os.makedirs(out_dir, exist_ok=True)
    for name in ("kbl_fp32_peaks", "kbl_int_fp64_rates"):
        src = os.path.join(here, "peaks", name + ".cu")
        exe = os.path.join(out_dir, name)
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-o", exe, src],
                       check=True)
        with ClockSampler(0) as clk:
            subprocess.run([exe], check=True)
        print(json.dumps({"peaks": name, "clocks": clk.summary()}), flush=True)


def main():
    args = parse()
    if args.peaks:
        run_peaks()
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank)), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    if args.workload == "adjoint":
        line, _, _ = run_adjoint(args, rank, world)
        if rank == 0:
            print(json.dumps(line), flush=True)
    elif args.workload == "triangles":
        import torch
        from paper_2407_20966_gb300 import build
        build.build()
        dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
        torch.cuda.set_device(dev)
        sub = run_triangles(args, steps=args.steps, warmup=args.warmup, dev=dev)
        if rank == 0:
            line = {"metric": METRIC, "value": sub["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                    "warmup": args.warmup, "ms_per_step": sub["ms_per_step"], "higher_is_better": True,
                    "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                    "config": {"workload": sub["workload"], "elements": sub["elements"], "l2": sub["l2"],
                               "parallelism": f"replicas x{world}"},
                    "e2e": sub["e2e"], "roofline": sub["roofline"], "clocks": sub["clocks"]}
            print(json.dumps(line), flush=True)
    elif args.workload == "batched":
        line, probs, _ = run_batched(args, rank, world)
        if rank == 0:
            if not args.no_cpu_baseline:
                line["cpu_baseline"] = oracle_batch_sample(probs, budget_s=12.0)
            print(json.dumps(line), flush=True)
    else:
        line, w0, wl = run_ours(args, rank, world)
        if args.workload == "vortex" and not args.no_subworkloads:
            # the larger configurations under the same clock: Sedov 512^2 P2 and the 4096-problem batch
            import torch
            dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
            line["sedov"] = run_sub_mesh(args, "sedov", steps=min(args.steps, 10), warmup=3, dev=dev)
            bl, _, _ = run_batched(args, rank, world, steps=3, warmup=1)
            line["batched"] = {k: bl[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup", "e2e",
                                                  "gpu_launches", "form", "roofline", "clocks")}
            line["batched"]["workload"] = bl["config"]["workload"]
            line["batched"]["elements"] = bl["config"]["elements"]
            line["batched"]["tuning"] = bl["config"]["tuning"]
            line["triangles"] = run_triangles(args, steps=min(args.steps, 10), warmup=3, dev=dev)
        if rank == 0:
            if not args.no_cpu_baseline:
                line["cpu_baseline"] = oracle_sample(args.workload, budget_s=12.0)
            print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
