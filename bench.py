"""Benchmark of the SPARKLING hot path on GB300.

One step = one projected-gradient iteration of full-3D SPARKLING over the
whole pattern (eq. proj_grad_descent / Algorithm 1 inner loop): pack, direct
attraction sum over the density grid, direct repulsion sum, combine, and the
per-shot projection with the gradient step fused in -- all through the C-ABI
entry point sparkling_step.

Metric: pair interactions per second, pairs = N*P + N*(N-1) per step
(directed attraction pairs with the P density points plus directed
repulsion pairs), with the seconds per iteration as ms_per_step.

Default workload: 4096 shots x 2560 samples = 10,485,760 samples, density
grid 256^3 = 16,777,216 points (the ~1e7-sample configuration).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload hr|diff|medium|small|tiny] [--acc kahan|fp64]

Under torchrun (N > 1) every rank runs an independent problem instance of
the same size (its own seed) on its own GPU: the trajectories are
independent problems, so there is no data-path collective; the ranks only
meet at the timing barriers and the max-over-ranks reduction.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time
from typing import Optional

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 512 << 20      # > 129 MB L2
SFU_RSQ_PER_SM_CLK = 16         # MUFU.RSQ results per SM per clock on GB300 (alu_peak_probe.cu)
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=("hr", "diff", "medium", "small", "tiny", "batched"),
                    default="hr")
    ap.add_argument("--path", choices=("kernels", "engine"), default="kernels",
                    help="single-trajectory step through sparkling_step (separate pair kernels) "
                         "or the persistent engine (sparkling_step_batched with B = 1)")
    ap.add_argument("--acc", choices=("kahan", "fp64"), default="kahan")
    ap.add_argument("--attraction", choices=("direct", "field"), default="direct",
                    help="direct sum (exact) or the interpolated node field of the density "
                         "(fast, approximate; the step's pairs are then counted as equivalent "
                         "pair interactions)")
    ap.add_argument("--repulsion", choices=("direct", "mesh"), default="direct",
                    help="every pair (exact) or the particle-particle particle-mesh summation "
                         "(fast, approximate; pairs counted as equivalent pair interactions)")
    ap.add_argument("--mesh-cells", type=int, default=512,
                    help="mesh cells across the sample box for --repulsion mesh")
    ap.add_argument("--mesh-sigma", type=float, default=2.0,
                    help="split width in mesh cells for --repulsion mesh")
    ap.add_argument("--mesh-rc", type=float, default=3.5,
                    help="short-range cut-off in split widths for --repulsion mesh")
    ap.add_argument("--shape-attraction", type=int, default=-1,
                    help="pin the attraction's tile shape (0/1/2: 128/256/512 threads; "
                         "-1: autotuned)")
    ap.add_argument("--shape-repulsion", type=int, default=-1,
                    help="pin the symmetric repulsion's tile shape (0: 2 sources per lane, "
                         "targets paired; 1: 4 sources, targets paired; 2: 2 sources, sources "
                         "paired; -1: autotuned)")
    ap.add_argument("--clock-log", default=None,
                    help="directory for the raw nvidia-smi clock samples (default: the temp dir)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target duration of the oracle sample")
    ap.add_argument("--crossover", action="store_true",
                    help="instead of the step: time the exact (symmetric) and the mesh repulsion "
                         "over a range of N and report where the mesh wins")
    a = ap.parse_args(argv)
    if a.steps is None:
        a.steps = 1 if a.workload == "hr" else 3
    if a.warmup < 3:
        ap.error("--warmup must be >= 3")
    if (a.attraction == "field" or a.repulsion == "mesh") and (a.workload == "batched"
                                                               or a.path == "engine"):
        ap.error("--attraction field / --repulsion mesh run on the kernels path "
                 "(the engine takes the direct sums)")
    return a


# --- distributed helpers (also exercised by the gloo tests) -------------------

def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def reduce_max(value: float, device=None) -> float:
    """Max of a scalar over all ranks (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# --- workload -----------------------------------------------------------------

def load_problem(name: str, seed: int):
    import inputs
    return inputs.make_problem(name, seed=seed)


def pairs_per_step(N: int, P: int) -> int:
    return N * P + N * (N - 1)


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, index: int, directory: Optional[str] = None):
        import tempfile
        self.index = index
        self.proc = None
        self.path = os.path.join(directory or tempfile.gettempdir(), f"clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={SMI_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def measure_probe():
    """Run alu_peak_probe.cu (built with nvcc) and return its per-SM-per-clock
    rates ({"rsqrt": .., "ffma": .., "dfma": .., "fp64acc": ..}), or {} when it
    cannot run."""
    import re
    import shutil
    import tempfile
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = os.path.join(ROOT, "alu_peak_probe.cu")
    if not (os.path.exists(nvcc) and os.path.exists(src)):
        return None
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "probe")
        r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                            src], capture_output=True, text=True)
        if r.returncode != 0:
            return {}
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    rates = {}
    for key, pat in (("rsqrt", r"^rsqrt\s"), ("ffma", r"^ffma\s"), ("attr_mix", r"^attr_mix"),
                     ("dfma", r"^dfma\s"), ("fp64acc", r"^fp64acc")):
        m = re.search(pat + r".*?ops/SM/clk = ([0-9.]+)", r.stdout, re.M)
        if m:
            rates[key] = float(m.group(1))
    return rates



# --- oracle timing (the CPU baseline and the reference arm) -------------------

def oracle_sample(prob, seconds: float, seed: int = 1):
    """Time the FP64 oracle on a bounded sample of targets of the workload;
    returns (pairs/s, description, threads)."""
    import numpy as np
    import oracle
    K = prob.K.astype(np.float64)
    N, P = K.shape[0], int(np.prod(prob.grid.n))
    rng = np.random.default_rng(seed)
    per_target = P + N - 1
    m = 2
    while True:
        idx = rng.choice(N, size=m, replace=False)
        t0 = time.perf_counter()
        oracle.forces(K, prob.grid, targets=idx)
        dt = time.perf_counter() - t0
        if dt >= seconds or m >= N:
            break
        if dt > 0.25:
            m = min(N, max(m + 1, int(m * seconds / dt * 1.05)))
        else:
            m = min(N, m * 4)
    pairs = m * per_target
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    desc = (f"{m} random targets of the {prob.name} workload, each against all "
            f"{P} density points and {N - 1} samples ({pairs:.3e} FP64 pairs, {dt:.1f} s)")
    return pairs / dt, desc, threads


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload == "batched":
        import inputs
        probs = inputs.make_batched(seed=0)
        prob = max(probs, key=lambda q: q.N)
        N = sum(q.N for q in probs)
        P = int(prob.grid.rho.size)
        pairs_step = sum(pairs_per_step(q.N, int(q.grid.rho.size)) for q in probs)
    else:
        prob = load_problem(args.workload, 0)
        N, P = prob.N, int(prob.grid.rho.size)
        pairs_step = pairs_per_step(N, P)
    vals = []
    desc = threads = None
    for _ in range(args.warmup):
        oracle_sample(prob, min(args.cpu_seconds, 3.0) / 3)
    for _ in range(args.steps):
        v, desc, threads = oracle_sample(prob, args.cpu_seconds / max(args.steps, 1))
        vals.append(v)
    value = statistics.median(vals)
    unit = "pairs/s"
    step_s = pairs_step / value
    out = {
        "impl": "reference", "metric": "pair_interactions_per_s", "value": value, "unit": unit,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {prob.recipe}", "N": N, "P": P,
                   "ms_per_step_note": "extrapolated from the sampled pair rate"},
        "cpu_baseline": {"value": value, "unit": unit, "cores": threads, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)
    return 0


# --- our implementation --------------------------------------------------------

class Workload:
    """Device state and the step call of one benchmark workload."""

    def __init__(self, sp, args, dev, seed):
        import torch
        self.sp, self.args, self.dev = sp, args, dev
        self.acc = sp.ACC_KAHAN32 if args.acc == "kahan" else sp.ACC_FP64
        if args.workload == "batched":
            import inputs
            self.probs = inputs.make_batched(seed=seed)
        else:
            self.probs = [load_problem(args.workload, seed)]
        self.batched = args.workload == "batched" or args.path == "engine"
        self.off = [0]
        for p in self.probs:
            self.off.append(self.off[-1] + p.N)
        self.Ns = self.probs[0].Ns
        self.K = torch.from_numpy(__import__("numpy").concatenate([p.K for p in self.probs])).to(dev)
        self.rhos = [torch.from_numpy(p.grid.rho).to(dev) for p in self.probs]
        self.grids = [sp.make_grid(r, p.grid.lo, p.grid.hi, p.grid.n)
                      for r, p in zip(self.rhos, self.probs)]
        self.projs = [sp.make_proj(p.proj.alpha, p.proj.beta, p.proj.box, p.proj.n_iter,
                                   p.proj.pin_index, p.proj.pin) for p in self.probs]
        self.etas = [p.eta for p in self.probs]
        self.pairs = sum(pairs_per_step(p.N, int(p.grid.rho.size)) for p in self.probs)
        self.N = self.off[-1]
        p0 = self.probs[0]
        if args.workload == "batched":
            self.desc = (f"batched: {len(self.probs)} trajectories, N_b = 512 x U{{32..512}} shots "
                         f"(total {self.N}), 64^3 Gaussian densities")
        else:
            self.desc = f"{args.workload}: {p0.recipe}"

    def step(self):
        sp = self.sp
        if self.batched:
            sp.sparkling_step_batched(self.ctx, self.K, self.off, self.Ns, self.grids, self.etas,
                                      self.projs, self.acc, graph=True)
        else:
            p = self.probs[0]
            sp.sparkling_step(self.ctx, self.K, p.Nc, p.Ns, self.grids[0], p.eta, self.projs[0],
                              self.acc)


def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2108_02991_gb300 as sp

    w = Workload(sp, args, dev, seed=rank)
    ctx = sp.sparkling_create(local)
    w.ctx = ctx
    if args.shape_attraction >= 0:
        sp.sparkling_set_shape(ctx, "attraction", args.shape_attraction)
    if args.shape_repulsion >= 0:
        sp.sparkling_set_shape(ctx, "repulsion", args.shape_repulsion)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    field_build_ms = None
    mesh_build_ms = None
    if args.repulsion == "mesh":
        sp.sparkling_set_repulsion(ctx, sp.REPULSION_MESH,
                                   sp.make_mesh(args.mesh_cells, args.mesh_sigma, args.mesh_rc))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        w.step()                                  # builds the kernel spectra (blocking)
        sp.sparkling_status(ctx)
        mesh_build_ms = (time.perf_counter() - t0) * 1e3
    if args.attraction == "field":
        sp.sparkling_set_attraction(ctx, sp.ATTRACTION_FIELD)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        sp.sparkling_attraction_field(ctx, w.grids[0])      # blocking
        field_build_ms = (time.perf_counter() - t0) * 1e3

    for _ in range(args.warmup):
        w.step()
    sp.sparkling_status(ctx)
    torch.cuda.synchronize(dev)

    sp.sparkling_set_timing(ctx, True)
    sp.sparkling_kernel_times(ctx, reset=True)
    launches0 = sp.sparkling_launch_count(ctx)
    clocks = ClockSampler(local, args.clock_log)
    clocks.start()
    barrier()
    torch.cuda.synchronize(dev)
    step_ms = []
    for _ in range(args.steps):
        flush.zero_()                        # evict L2 between timed steps (not timed)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        w.step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    sp.sparkling_status(ctx)
    launches = sp.sparkling_launch_count(ctx) - launches0
    ktimes = sp.sparkling_kernel_times(ctx, reset=True)
    sp.sparkling_set_timing(ctx, False)

    local_ms = sum(step_ms)
    total_ms = reduce_max(local_ms, dev)
    pairs_all = reduce_sum(float(w.pairs * args.steps), dev)
    value = pairs_all / (total_ms * 1e-3)

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    probe = measure_probe() if rank == 0 else {}
    rsq = probe.get("rsqrt")
    rate = float(round(rsq)) if rsq else float(SFU_RSQ_PER_SM_CLK)
    peak = sms * rate * max_mhz * 1e6
    if w.batched:
        # one engine launch runs every pair of the step: N_b*P_b + N_b*(N_b-1)
        kname, kpairs = "engine", w.pairs
    elif args.repulsion == "mesh" and args.attraction == "direct":
        p0 = w.probs[0]
        kname, kpairs = "attraction", p0.N * int(p0.grid.rho.size)
    elif args.attraction == "field" and args.repulsion == "direct":
        # the attraction is an interpolation; the symmetric repulsion takes
        # one reciprocal square root per unordered pair
        kname, kpairs = "repulsion", w.N * (w.N - 1) // 2
    elif args.attraction == "field":
        kname, kpairs = None, None
    else:
        p0 = w.probs[0]
        kname, kpairs = "attraction", p0.N * int(p0.grid.rho.size)
    k_ms, k_n = ktimes[kname] if kname else (0.0, 0)
    achieved = kpairs / (k_ms / k_n * 1e-3) if k_n else None
    roof = {"bound": "alu", "achieved": achieved / 1e9 if achieved else None,
            "peak": peak / 1e9, "unit": "Gpair/s",
            "frac": (achieved / peak) if achieved else None, "traffic": None,
            "kernel": kname,
            "peak_basis": f"{sms} SMs x {rate:g} MUFU.RSQ/clk/SM x {max_mhz:.0f} MHz max SM clock "
                          f"(one reciprocal square root per pair; probe measured "
                          f"{rsq if rsq else 'n/a'} RSQ/clk/SM)"}
    if clk and achieved:
        roof["frac_at_measured_clock"] = achieved / (sms * rate * clk["sm_mhz"] * 1e6)
    tot_k = max(sum(v[0] for v in ktimes.values()), 1e-9)
    kernels = {k: {"ms_total": round(ms, 3), "launches": n, "share": round(ms / tot_k, 4)}
               for k, (ms, n) in ktimes.items() if n}
    if not w.batched and ktimes["repulsion"][1]:
        rep_ms, rep_n = ktimes["repulsion"]
        kernels["repulsion"]["gpair_per_s"] = w.N * (w.N - 1) / (rep_ms / rep_n * 1e-3) / 1e9

    e2e = None
    if not args.no_e2e and not w.batched:
        p = w.probs[0]
        Kh = torch.from_numpy(p.K).pin_memory()
        rhoh = torch.from_numpy(p.grid.rho).pin_memory()
        hgrid = sp.make_grid(rhoh, p.grid.lo, p.grid.hi, p.grid.n)
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sp.sparkling_step_host(ctx, Kh, p.Nc, p.Ns, hgrid, rhoh, p.eta, w.projs[0], w.acc)
        t1 = time.perf_counter()
        barrier()
        e2e_s = reduce_max(t1 - t0, dev)
        e2e = {"value": pairs_all / e2e_s, "unit": "pairs/s",
               "h2d_bytes_per_step": int(Kh.numel() * Kh.element_size() + rhoh.numel() * 4),
               "d2h_bytes_per_step": int(Kh.numel() * Kh.element_size())}
    elif not args.no_e2e:
        # batched: pinned host copy of K in and out around every step
        Kh = w.K.cpu().pin_memory()
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            w.K.copy_(Kh, non_blocking=True)
            w.step()
            Kh.copy_(w.K, non_blocking=True)
            torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        barrier()
        e2e_s = reduce_max(t1 - t0, dev)
        nb = int(Kh.numel() * Kh.element_size())
        e2e = {"value": pairs_all / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": nb, "note": "densities resident on the device"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, desc, threads = oracle_sample(w.probs[0], args.cpu_seconds)
        cpu = {"value": v, "unit": "pairs/s", "cores": threads, "kind": "oracle", "sample": desc}

    if rank == 0:
        p0 = w.probs[0]
        out = {
            "metric": "pair_interactions_per_s", "value": value, "unit": "pairs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32 pairs, " + ("compensated-f32" if w.acc == 0 else "f64")
                     + " per-target sums, f64 projection",
            "data": "synthetic",
            "config": {"workload": w.desc, "N": w.N, "P": int(p0.grid.rho.size),
                       "trajectories": len(w.probs), "Ns": w.Ns, "pairs_per_step": w.pairs,
                       "n_pit": p0.proj.n_iter, "path": "engine" if w.batched else "kernels",
                       "l2": "flushed (512 MB write) between timed steps", "acc": args.acc,
                       "attraction": args.attraction, "repulsion": args.repulsion,
                       "shapes": ("autotuned" if args.shape_attraction < 0
                                  and args.shape_repulsion < 0 else
                                  f"pinned: attraction {args.shape_attraction}, "
                                  f"repulsion {args.shape_repulsion} (-1: autotuned)")},
            "roofline": roof, "kernels": kernels, "clocks": clk, "e2e": e2e,
            "cpu_baseline": cpu, "gpu_launches": launches,
            "seconds_per_iteration": total_ms / args.steps / 1e3,
            "autotuner": [l for l in sp.sparkling_tuning_report(ctx).splitlines() if l],
            "alu_probe_per_sm_clk": probe or None,
        }
        if mesh_build_ms is not None:
            out["mesh"] = {
                "cells": args.mesh_cells, "sigma_cells": args.mesh_sigma,
                "rc_sigmas": args.mesh_rc, "first_step_ms": mesh_build_ms,
                "note": "particle-particle particle-mesh repulsion; the first step builds the "
                        "kernel spectra once; value counts N*P + N*(N-1) equivalent pairs"}
        if field_build_ms is not None:
            out["field"] = {
                "build_ms": field_build_ms,
                "note": "node field of the density (FP64 FFT convolution, once per density, "
                        "outside the timed steps); value counts N*P + N*(N-1) equivalent pairs; "
                        "the e2e leg rebuilds the field every step (the density is copied in)"}
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_crossover(args):
    """Repulsion-only timing of the exact symmetric kernel and of the mesh
    summation (sigma 2.5 cells, cut-off 4 sigma, mesh cells growing like
    N^(1/3), 256 at 10.5M samples) on uniform samples in [-0.45, 0.45]^3; the
    mesh result is compared with the exact one computed on the device."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2108_02991_gb300 as sp
    import inputs
    dev = torch.device("cuda", 0)
    grid = inputs.density_gaussian(8, 0.2)
    rho = torch.from_numpy(grid.rho).to(dev)
    g = sp.make_grid(rho, grid.lo, grid.hi, grid.n)
    rows = []
    for N in (10_000, 30_000, 100_000, 300_000, 1_000_000, 3_000_000):
        K = torch.from_numpy(np.random.default_rng(N).uniform(-0.45, 0.45, size=(N, 3))
                             .astype(np.float32)).to(dev)
        cells = int(min(512, max(16, round(256 * (N / 10_485_760) ** (1 / 3) / 8) * 8)))
        out = {}
        for mode in ("direct", "mesh"):
            ctx = sp.sparkling_create(0)
            if mode == "mesh":
                sp.sparkling_set_repulsion(ctx, sp.REPULSION_MESH, sp.make_mesh(cells))
            R = torch.empty(N, 3, dtype=torch.float64, device=dev)
            G = torch.empty_like(R)
            for _ in range(2):                   # tuning / kernel spectra, then warm
                sp.sparkling_grad(ctx, K, g, sp.ACC_KAHAN32, G=G, R=R)
            sp.sparkling_status(ctx)
            sp.sparkling_set_timing(ctx, True)
            sp.sparkling_kernel_times(ctx, reset=True)
            for _ in range(args.steps):
                sp.sparkling_grad(ctx, K, g, sp.ACC_KAHAN32, G=G, R=R)
            sp.sparkling_status(ctx)
            ms, n = sp.sparkling_kernel_times(ctx, reset=True)["repulsion"]
            out[mode] = (ms / n, R.clone())
            ctx.close()
        err = float(torch.linalg.norm(out["mesh"][1] - out["direct"][1]) /
                    torch.linalg.norm(out["direct"][1]))
        rows.append({"N": N, "mesh_cells": cells, "direct_ms": out["direct"][0],
                     "mesh_ms": out["mesh"][0], "mesh_rel_l2_vs_direct": err})
    cross = next((r["N"] for r in rows if r["mesh_ms"] < r["direct_ms"]), None)
    print(json.dumps({"metric": "repulsion_crossover", "unit": "ms per repulsion evaluation",
                      "rows": rows, "first_N_where_mesh_is_faster": cross,
                      "data": "synthetic: uniform samples in [-0.45, 0.45]^3"}), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.crossover:
        return run_crossover(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
