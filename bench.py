"""Benchmark of the coupled fluid + solute lattice-Boltzmann step on GB300.

Workload: the miscible layered anisotropic medium, 128^3 cells, FP32
population storage, solute inlet/outlet, linear hardening viscosity (the
fused per-cell update of the paper's Sections 2-4). Every step accumulates
the inlet/outlet solute flux in FP64 and checks that each warp's mass and
solute sums are finite; the FP64 mass and solute totals are formed by
lb_reduce in the end-to-end leg. One "step" = one lattice update of every
cell.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line. Under torchrun each rank advances its own replica of
the domain (weak scaling, no data-path collective); rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = NY = NZ = 128
ALGO_BYTES_PER_LUP = 321  # f 152 + h 152 + eps 4 + K^-1 12 + solid mask 1 (FP32 storage)
METRIC = "coupled LB MLUPS"
WORKLOAD = ("miscible porous medium 128^3, D3Q19 fluid + D3Q19 solute, diagonal anisotropic K, "
            "linear hardening tau(C), solute inlet/outlet; every step: FP64 accumulation of the "
            "inlet/outlet flux and a finite check of each warp's mass and solute sums")
PROFILE_JSON = os.path.join(ROOT, "profiles", "step_kernel_miscible128_traffic.json")

# Other workloads timed the same way (--workload); the default line is "miscible".
# name: (factory(rank), storage, algorithmic bytes per cell update, description)
def _other_workloads():
    from paper_0912_4230_gb300 import workloads as W
    prec = "precision porous medium 256^3, full SPD K per 32^3 block, D3Q19 fluid + solute, "
    return {
        "precision-fp32": (lambda r: W.precision(seed=r, storage="fp32"), "fp32", 333,
                           prec + "FP32 storage"),
        "precision-fp16": (lambda r: W.precision(seed=r, storage="fp16"), "fp16", 181,
                           prec + "FP16 deviation storage"),
        "precision-bf16": (lambda r: W.precision(seed=r, storage="bf16"), "bf16", 181,
                           prec + "BF16 deviation storage"),
        "plain-fp64": (lambda r: W.plain_channel(), "fp64", 337,
                       "plain Brinkman channel 16x16x64, FP64, no solute"),
        # algorithmic bytes: f and three solute lattices read and written once,
        # eps, K^-1 and the mask read once
        "species": (lambda r: W.miscible_species(seed=r), "fp32", 4 * 152 + 17,
                    "miscible medium 128^3 with three solute species (tau_D 0.8 / 1.2 / 0.6), "
                    "D3Q19 fluid + 3 solute lattices, FP32; one fused pass per step"),
        "wood": (lambda r: W.wood(nx=256, ny=192, nz=64, wood_depth=128), "fp32", 333,
                 "adhesive pressed into wood 256x192x64 (year rings of 30 cells at 45 deg, "
                 "full SPD K, pressure faces, solute inlet/outlet, hardening law), FP32"),
        "forchheimer": (lambda r: W.forchheimer(seed=r), "fp32", 321,
                        "coarse porous medium 128^3 with Forchheimer drag (diagonal K, "
                        "K_zz = 10 K_xx, G 1e-4), D3Q19 fluid + solute, FP32"),
        # free surface: algorithmic bytes counted per updated (liquid or interface) cell
        "drop": (lambda r: W.drop(seed=r), "fp32", 171,
                 "free-surface drop 192x192x128 (R 24, 40 cells above a solid wall), A 1e-3, "
                 "FP32, five passes over the active tiles per step; roofline per updated cell"),
    }


def kernel_source_hash() -> str:
    """Hash of the code (comments and blank lines dropped) of the sources that
    define and launch the benchmarked step kernel: a recorded capture stays
    valid across comment edits and lapses with any code change."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_0912_4230_gb300", "csrc")
    for f in ("lb_common.cuh", "lb_kernels.cuh", "lb_inst.cuh"):
        src = open(os.path.join(csrc, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in src.splitlines()]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


class NvmlClocks:
    """SM clock and clock-event reasons read through NVML (libnvidia-ml,
    read-only queries) as often as the host can while the timed launches run,
    so that a timed region of a few milliseconds still has samples."""

    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
            "hw_thermal_slowdown": 0x40}

    def __init__(self, index: int):
        import ctypes
        self.samples = []
        self.ok = False
        try:
            L = ctypes.CDLL("libnvidia-ml.so.1")
            if L.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            if L.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h)) != 0:
                return
            self.L, self.ct = L, ctypes
            self.reasons_fn = getattr(L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(L, "nvmlDeviceGetCurrentClocksThrottleReasons")
            mx = ctypes.c_uint()
            self.max_mhz = float(mx.value) if L.nvmlDeviceGetMaxClockInfo(
                self.h, ctypes.c_int(1), ctypes.byref(mx)) == 0 else None
            self.ok = True
        except (OSError, AttributeError):
            self.ok = False

    def sample(self):
        if not self.ok:
            return
        ct = self.ct
        mhz, bits = ct.c_uint(), ct.c_ulonglong()
        if (self.L.nvmlDeviceGetClockInfo(self.h, ct.c_int(1), ct.byref(mhz)) == 0 and
                self.reasons_fn(self.h, ct.byref(bits)) == 0):
            self.samples.append((float(mhz.value), int(bits.value)))

    def summary(self):
        if not self.samples:
            return None
        reasons = sorted({n for n, b in self.BITS.items() for _, r in self.samples if r & b})
        return {"sm_mhz": statistics.median(m for m, _ in self.samples),
                "sm_max_mhz": self.max_mhz, "reasons": reasons, "samples": len(self.samples),
                "source": "NVML during the timed region"}


def clocks_record(nvml, smi):
    """The line's clock record: NVML samples taken during the timed launches
    when there are any, else nvidia-smi's over warm-up and timed region."""
    s = nvml.summary() if nvml is not None else None
    if s is None:
        s = dict(smi.summary())
        s["source"] = "nvidia-smi over warm-up and timed region"
    elif s["sm_max_mhz"] is None:
        s["sm_max_mhz"] = smi.summary().get("sm_max_mhz")
    return s


def nvml_index(local: int) -> int:
    """NVML's index of this process's CUDA device (CUDA_VISIBLE_DEVICES may
    renumber it)."""
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v.strip() for v in vis.split(",") if v.strip()]
    if ids and all(v.isdigit() for v in ids) and local < len(ids):
        return int(ids[local])
    return local


def workload_config(ws: int, workload: str, N: int, lattice, algo: int) -> dict:
    """The config of a bench line; both arms print the same one."""
    return {"workload": workload, "cells": N, "lattice": list(lattice),
            "parallelism": f"replicas{ws}",
            "l2": f"inputs larger than L2: {algo * N / 1e6:.0f} MB moved per step"}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v: float, device: str = "cuda") -> float:
    """The largest value over all ranks (timings: the job is as slow as its
    slowest replica)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws: int, cells_per_rank: int, steps: int, seconds_max: float) -> float:
    """Whole-job MLUPS of ws replicas (weak scaling): every rank advances its
    own lattice, the job takes as long as the slowest rank."""
    return ws * cells_per_rank * steps / seconds_max / 1e6


def cpu_baseline(prob, budget_s: float = 12.0):
    """The FP64 oracle on this host's cores, on a bounded sample of the
    workload: the full lattice for as many steps as fit the budget."""
    from oracle import oracle as O
    threads = os.cpu_count() or 1
    o = O.Oracle(prob, threads=threads)
    t0 = time.perf_counter()
    o.step(1)
    one = time.perf_counter() - t0
    steps = max(1, min(50, int(budget_s / max(one, 1e-3))))
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return {"value": prob.N * steps / dt / 1e6, "unit": "MLUPS", "cores": threads,
            "kind": "oracle",
            "sample": f"full {prob.nx}x{prob.ny}x{prob.nz} lattice, {steps} steps after 1 warm-up "
                      f"step, FP64, OpenMP over {threads} threads"}


def run_reference(args):
    """The oracle as the reference arm: K timed steps (after W warm-up) on a
    bounded sample of the workload, on the host cores."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_0912_4230_gb300 import workloads as W
    threads = os.cpu_count() or 1
    prob = W.miscible(NX, NY, NZ, seed=0)
    o = O.Oracle(prob, threads=threads)
    t0 = time.perf_counter()
    o.step(1)
    one = time.perf_counter() - t0
    # bound the whole run to about two minutes: crop the lattice in z if needed
    budget = 120.0
    nz = NZ
    est = one * (args.steps + args.warmup)
    if est > budget:
        nz = max(4, int(NZ * budget / est))
        prob = W.crop(prob, 0, 0, 0, NX, NY, nz)
        o = O.Oracle(prob, threads=threads)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    v = prob.N * args.steps / dt / 1e6
    sample = f"{NX}x{NY}x{nz} lattice (of {NX}x{NY}x{NZ}), {args.steps} steps, FP64"
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3 * (NZ / nz),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(ws, WORKLOAD, NX * NY * NZ, (NX, NY, NZ), ALGO_BYTES_PER_LUP),
        "arm": "FP64 CPU oracle (plain, cell by cell) on the host cores",
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def mix_kernel_rate(stream, storage: str, per_class: int = 3, steps: int = 200) -> dict:
    """The step kernel's own MLUPS on the serving mix, the yardstick of the
    serving loop's throughput: for each side class, a few of the stream's
    lattices each stepped alone (one lb_step call of `steps` steps after a
    warm-up, CUDA graphs on, timed with CUDA events on its stream); the mix
    rate weights each class's mean time per lattice update by the lattice
    updates the whole stream asks of that class."""
    import torch
    from paper_0912_4230_gb300 import lb, workloads as W
    s = torch.cuda.current_stream()
    by_side = {}
    for q in stream:
        by_side.setdefault(q["nx"], []).append(q)
    rate, total_lup, total_s = {}, 0.0, 0.0
    for side, qs in sorted(by_side.items()):
        secs = []
        for q in qs[:per_class]:
            p = W.request_problem(q, storage=storage)
            g = lb.Lattice(p, storage=storage, kernel="cell", stream=s.cuda_stream)
            g.step(21)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            g.step(steps)
            e1.record(s)
            e1.synchronize()
            secs.append(e0.elapsed_time(e1) * 1e-3 / (steps * p.N))   # s per lattice update
            g.close()
        per_lup = sum(secs) / len(secs)
        lup = sum(q["nx"] * q["ny"] * q["nz"] * q["steps"] for q in qs)
        rate[str(side)] = 1e-6 / per_lup
        total_lup += lup
        total_s += lup * per_lup
    return {"mlups": total_lup / total_s / 1e6, "by_side_mlups": rate,
            "how": f"per side class up to {per_class} of the stream's lattices stepped alone "
                   f"for {steps} steps, weighted by the stream's lattice updates"}


def run_serving(args):
    """Serving workload: a Poisson stream of miscible-medium solves of sizes
    32..160 (z-aspect up to 2) under a 120 GB HBM budget, steps scaled down so
    that the run takes seconds; continuous batching (FP32 and FP16 storage)
    against the plain per-lattice FP32 path (one request at a time)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_0912_4230_gb300 import serve, workloads as W
    from paper_0912_4230_gb300 import lb
    n_req, scale = args.requests, args.steps_scale
    stream = W.requests(n=n_req, rate=50.0, seed=5)
    # every lattice is sub-allocated from one packed arena of the admission
    # budget inside a torch tensor: no cudaMalloc/cudaFree per request
    budget = 120 * 10 ** 9
    region = torch.empty(budget, dtype=torch.uint8, device="cuda")
    arena = lb.Arena(budget, region.data_ptr())
    arena.use()
    step_s, admit_s = torch.cuda.Stream(), torch.cuda.Stream()
    res = {}
    cap = args.max_resident or None
    arms = [a for a in (("batched_fp32", "fp32", True, cap),
                        ("batched_fp16", "fp16", True, cap),
                        ("per_lattice_fp32", "fp32", False, 1))
            if a[0] in args.arms.split(",")]
    kernel = {st: mix_kernel_rate(stream, st) for st in sorted({a[1] for a in arms})}
    for name, storage, batched, maxres in arms:
        reqs = serve.make_requests(stream, storage=storage, steps_scale=scale)
        be = serve.LibraryBackend(storage, keep_fields=False, batched=batched,
                                  admit_stream=admit_s, step_stream=step_s)
        srv = serve.Server(be, budget_bytes=budget, chunk=args.chunk, max_resident=maxres,
                           fill_cells=(args.fill_cells or None) if batched else None,
                           admit_in_thread=True)
        torch.cuda.synchronize()
        with ClockSampler(0) as clk:
            st = srv.run(reqs)
            torch.cuda.synchronize()
        st["clocks"] = clk.summary()
        st["arena_peak_bytes"] = arena.stats()["peak"]
        st["chunks"] = len(srv.log)
        st["mean_cells_stepped"] = (sum(e["stepped_cells"] for e in srv.log) / len(srv.log)
                                    if srv.log else 0)
        st["of_kernel_mix_rate"] = st["mlups"] / kernel[storage]["mlups"]
        res[name] = st
    lb.Arena.use_none()
    arena.close()
    del region
    b = res[arms[0][0]]
    line = {
        "metric": "served-solve throughput (MLUPS) and p50/p99 latency", "value": b["mlups"],
        "unit": "MLUPS", "n_gpus": 1, "steps": sum(r.steps for r in serve.make_requests(stream, steps_scale=scale)),
        "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{n_req} requests, Poisson 50/s, sides 32..160, z-aspect 1..2, "
                               f"steps U(2000, 20000) x {scale}, 120 GB admission budget (one packed arena), "
                               f"chunk {args.chunk} steps, at most "
                               f"{args.max_resident or 'budget-many'} resident, oldest stepped "
                               f"together up to {args.fill_cells or 'all'} cells"},
        "serving": res,
        "kernel_mix_rate": kernel,
        "gpu_launches": None,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-iters", type=int, default=5)
    ap.add_argument("--e2e-inner", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="miscible")
    ap.add_argument("--kernel", default="auto", choices=["auto", "cell", "rows", "staged"])
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--graphs", default="on", choices=["on", "off"],
                    help="replay step pairs from a CUDA graph (on) or launch every step")
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--arms", default="batched_fp32,batched_fp16,per_lattice_fp32",
                    help="serving: the arms to run, comma-separated")
    ap.add_argument("--steps-scale", type=float, default=0.02)
    ap.add_argument("--chunk", type=int, default=100)
    ap.add_argument("--max-resident", type=int, default=0,
                    help="serving: cap on resident lattices (0 = HBM budget only)")
    ap.add_argument("--fill-cells", type=int, default=4 * 1024 * 1024,
                    help="serving: step the oldest lattices until this many cells (0 = all)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)

    import torch
    import __graft_entry__
    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if rank == 0:
        __graft_entry__.build()
    barrier(ws)
    from paper_0912_4230_gb300 import lb, workloads as W

    algo, workload, storage = ALGO_BYTES_PER_LUP, WORKLOAD, "fp32"
    if args.workload == "miscible":
        prob = W.miscible(NX, NY, NZ, seed=rank)
    else:
        fac, storage, algo, workload = _other_workloads()[args.workload]
        prob = fac(rank)
        args.no_cpu_baseline = True
    stream = torch.cuda.current_stream()
    lat = lb.Lattice(prob, storage=storage, check_every=1, stream=stream.cuda_stream,
                     kernel=args.kernel)
    N = prob.N
    choice = 0
    if not args.no_autotune and args.kernel == "auto":
        choice = lb.lb_autotune(lat.ctx, 5)   # launch shape picked by timing, state unchanged
    if args.graphs == "off":
        lat.set_graphs(False)
    # one call, so that a CUDA graph of the step pair is captured before timing
    K = args.steps
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nvml = NvmlClocks(nvml_index(local))
    with ClockSampler(local) as clk:   # nvidia-smi over warm-up and the timed region
        lat.step(args.warmup)
        torch.cuda.synchronize()
        barrier(ws)
        torch.cuda.synchronize()
        # K steps in one lb_step call: K launches of the step kernel (the
        # fields are exported by the last one only), nothing else on the stream
        nvml.sample()
        start.record(stream)
        lat.step(K)
        stop.record(stream)
        while not stop.query():       # NVML samples while the launches run
            nvml.sample()
        torch.cuda.synchronize()
    barrier(ws)
    total_ms = start.elapsed_time(stop)
    # the step kernel is the only launch in the region (the free-surface step:
    # its six kernels), so its average launch duration is at most the region's
    # time over K; that bound (launch gaps included) is what the roofline uses
    kern_ms = total_ms / K
    lat.sync()  # raises on a non-finite reduction
    total_ms = max_over_ranks(ws, total_ms)
    kern_ms = max_over_ranks(ws, kern_ms)
    ms_per_step = total_ms / K
    value = job_value(ws, N, K, total_ms * 1e-3)

    # end to end through the C ABI with host buffers: upload the initial
    # fields, advance, read the fields and totals back
    rho0 = torch.from_numpy(prob.rho0).pin_memory()
    u0 = torch.from_numpy(prob.u0).pin_memory()
    C0 = torch.from_numpy(prob.C0).pin_memory() if prob.C0 is not None else None
    ctype = torch.from_numpy(prob.cell_type).pin_memory() if prob.cell_type is not None else None
    lam0 = torch.from_numpy(prob.lambda0).pin_memory() if prob.lambda0 is not None else None
    out = [torch.empty(n, dtype=torch.float32).pin_memory() for n in (N, 3 * N, N, N)]
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.e2e_iters):
        lb.lb_init(lat.ctx, rho0, u0, C0, ctype, lam0)
        lb.lb_step(lat.ctx, args.e2e_inner)
        lb.lb_fields(lat.ctx, *out)
        lb.lb_reduce(lat.ctx)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(ws, time.perf_counter() - t0)
    e2e_val = ws * N * args.e2e_inner * args.e2e_iters / e2e_s / 1e6
    # copies of one end-to-end iteration (inputs up, fields and totals down),
    # reported per lattice step of it
    h2d_iter = (5 if C0 is not None else 4) * N * 4 + (N * 5 if ctype is not None else 0)
    d2h_iter = 6 * N * 4 + 4 * 8
    h2d, d2h = h2d_iter / args.e2e_inner, d2h_iter / args.e2e_inner

    peak, peak_kind = measured_peaks()
    species = int(prob.params.get("species", 1))
    # launches of one step: the free surface's five passes; else the fused
    # step (which also advances further solute species), plus the density
    # pre-pass with surface tension
    if prob.cell_type is not None:
        launches_per_step = 5
    else:
        launches_per_step = 1 + (1 if prob.params.get("A", 0.0) else 0)
    units = N
    if prob.cell_type is not None:
        units = int(((prob.cell_type != W.EMPTY) & (prob.solid == 0)).sum())  # updated cells
    achieved = algo * units / (kern_ms * 1e-3) / 1e9
    traffic = None
    if os.path.exists(PROFILE_JSON) and args.workload == "miscible":
        pj = json.load(open(PROFILE_JSON))
        if pj.get("source_hash") == kernel_source_hash():
            traffic = pj.get("dram_bytes_per_launch")
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline(W.miscible(NX, NY, NZ, seed=0))
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "fp16": "f32 (f16 storage)",
                  "bf16": "f32 (bf16 storage)"}[storage], "data": "synthetic",
        "config": workload_config(ws, workload, N, (prob.nx, prob.ny, prob.nz), algo),
        "storage": storage, "cuda_graphs": args.graphs,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": peak_kind,
                     "kernel": ("five free-surface launches of one step" if prob.cell_type is not None
                                else "step_kernel (fluid and every solute species)"
                                if species > 1 else
                                "tma_step_kernel (row-pipelined)" if choice == 256 else
                                f"pipe_step_kernel (row-staged), rows of {choice - 1000} threads"
                                if choice > 1000 else
                                f"step_kernel, rows of {choice or 'default'} threads"),
                     "kernel_ms_from": "CUDA events around the K launches / K",
                     "kernel_ms": kern_ms, "algorithmic_bytes_per_lup": algo,
                     "units_per_step": units},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "step": f"lb_init from pinned host fields + {args.e2e_inner} lattice steps + "
                        f"lb_fields to pinned host + lb_reduce; bytes per lattice step (one "
                        f"iteration's {h2d_iter} B up and {d2h_iter} B down over its "
                        f"{args.e2e_inner} steps)"},
        "gpu_launches": K * launches_per_step,
        "clocks": clocks_record(nvml, clk),
    }
    print(json.dumps(line), flush=True)
    lat.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
