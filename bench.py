"""Benchmark of the SPARKLING hot path on GB300.

One step = one projected-gradient iteration of full-3D SPARKLING over the
whole pattern (eq. proj_grad_descent / Algorithm 1 inner loop): pack, direct
attraction sum over the density grid, direct repulsion sum, combine, and the
per-shot projection with the gradient step fused in -- all through the C-ABI
entry point sparkling_step_host, which copies the pattern and the density in
from pinned host memory, steps, and copies the pattern back.

Every warm-up and timed step is one such call.  In the timed steps the
library brackets the device work of the step (after the input copies, before
the output copy) with CUDA events on the launch stream: pairs / that time is
`value` (inputs resident in HBM); pairs / the wall time of the whole call is
`e2e` (host copies included).

Metric: pair interactions per second, pairs = N*P + N*(N-1) per step
(directed attraction pairs with the P density points plus directed
repulsion pairs), with the seconds per iteration as ms_per_step.

Default workload: 4096 shots x 2560 samples = 10,485,760 samples, density
grid 256^3 = 16,777,216 points (the ~1e7-sample configuration).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload hr|diff|medium|small|tiny|batched]
                  [--acc kahan|fp64|fp64pair] [--projection fp64|mixed]

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
    ap.add_argument("--path", choices=("auto", "kernels", "engine"), default="auto",
                    help="device path of the single-trajectory step (sparkling_set_step_path): "
                         "the library's choice (the persistent engine from 2^22 samples on), the "
                         "separate kernels, or the one-launch persistent engine")
    ap.add_argument("--acc", choices=("kahan", "fp64", "fp64pair"), default="kahan",
                    help="per-target accumulation: compensated FP32 folds, FP64 folds, or the "
                         "plain FP64-accumulate form (every attraction pair term added in FP64)")
    ap.add_argument("--trajectories", type=int, default=64,
                    help="batched workload: keep the first B of its 64 trajectories (a smaller "
                         "launch of the same kernels, e.g. for a profiler capture)")
    ap.add_argument("--two-launches", action="store_true",
                    help="batched step: the symmetric repulsion in its own kernel ahead of the "
                         "engine instead of as items of the engine's work list (one launch)")
    ap.add_argument("--projection", choices=("fp64", "mixed"), default="fp64",
                    help="projection arithmetic: FP64 duals (default) or the opt-in mixed form")
    ap.add_argument("--shot-stride", type=int, default=1,
                    help="keep every S-th shot of the workload (same density): a smaller launch "
                         "of the same kernels, e.g. for a profiler capture")
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
                    help="pin the symmetric repulsion's tile shape (256 threads: 0: 2 sources "
                         "per lane, targets paired; 1: 4 sources, targets paired; 2: 2 sources, "
                         "sources paired; 128 threads: 3: 8 targets and 2 sources per lane, "
                         "sources paired; -1: autotuned)")
    ap.add_argument("--clock-log", default=None,
                    help="directory for the raw nvidia-smi clock samples (default: the temp dir)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="target duration of the oracle sample")
    ap.add_argument("--crossover", action="store_true",
                    help="instead of the step: time the exact (symmetric) and the mesh repulsion "
                         "over a range of N and report where the mesh wins")
    a = ap.parse_args(argv)
    if a.steps is None:
        a.steps = 1 if a.workload == "hr" else 3
    if a.warmup < 3:
        ap.error("--warmup must be >= 3")
    if (a.attraction == "field" or a.repulsion == "mesh") and a.workload == "batched":
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

def load_problem(name: str, seed: int, shot_stride: int = 1):
    import inputs
    p = inputs.make_problem(name, seed=seed)
    if shot_stride > 1:
        Nc = (p.Nc + shot_stride - 1) // shot_stride
        p.K = p.K.reshape(p.Nc, p.Ns, 3)[::shot_stride].reshape(-1, 3).copy()
        p.Nc = Nc
        p.recipe += f"; every {shot_stride}th shot ({Nc} shots)"
        p.eta = 1.0 / p.N if p.eta else p.eta
    return p


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



# --- DRAM traffic of the attraction launch (from a committed ncu summary) ------

TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "attraction_hr_traffic.md")
ATTRACTION_SOURCES = ("pair_dev.cuh", "pairs.cu", "ptx.cuh", "kernels.h")


def attraction_source_sha() -> str:
    """SHA-256 (16 hex digits) of the attraction kernel's source files."""
    import hashlib
    h = hashlib.sha256()
    for name in ATTRACTION_SOURCES:
        with open(os.path.join(ROOT, "paper_2108_02991_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def attraction_traffic(prob, args):
    """DRAM bytes per attraction launch of this workload, from the ncu
    summary's linear fit in the number of targets (captured on launches of
    the same density with fewer shots); None unless the summary exists, was
    taken on the current kernel source and covers this workload's density."""
    import re
    try:
        text = open(TRAFFIC_PROFILE).read()
    except OSError:
        return None
    m = re.search(r"traffic-fit:\s*kernel_sha=(\w+)\s+density=(\d+)\s+"
                  r"bytes_const=([0-9.eE+]+)\s+bytes_per_target=([0-9.eE+]+)", text)
    if not m or m.group(1) != attraction_source_sha() or args.acc != "kahan":
        return None
    if int(m.group(2)) != int(prob.grid.rho.size):
        return None
    b = float(m.group(3)) + float(m.group(4)) * prob.N
    return {"bytes_per_launch": b,
            "basis": f"ncu dram__bytes_read.sum + dram__bytes_write.sum of launches with the same "
                     f"density and fewer shots, fitted linearly in the targets "
                     f"({os.path.relpath(TRAFFIC_PROFILE, ROOT)}, kernel source {m.group(1)})"}


# --- oracle timing (the CPU baseline and the reference arm) -------------------

def oracle_threads() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def oracle_sample(prob, seconds: float, seed: int = 1, K64=None):
    """Time the FP64 oracle on a bounded sample of targets of the workload:
    first 4 targets per core (every core busy), then, if that took less than
    `seconds`, a sample scaled to take about `seconds`.  Returns
    (pairs/s, description, threads)."""
    import numpy as np
    import oracle
    K = prob.K.astype(np.float64) if K64 is None else K64
    N, P = K.shape[0], int(np.prod(prob.grid.n))
    rng = np.random.default_rng(seed)
    per_target = P + N - 1
    threads = oracle_threads()
    m = min(N, 4 * threads)
    for attempt in range(3):
        idx = rng.choice(N, size=m, replace=False)
        t0 = time.perf_counter()
        oracle.forces(K, prob.grid, targets=idx)
        dt = time.perf_counter() - t0
        if attempt == 2 or dt >= 0.7 * seconds or m >= N:
            break
        m = min(N, max(m, int(m * seconds / max(dt, 1e-6))))
    pairs = m * per_target
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
        prob = load_problem(args.workload, 0, args.shot_stride)
        N, P = prob.N, int(prob.grid.rho.size)
        pairs_step = pairs_per_step(N, P)
    import numpy as np
    K64 = prob.K.astype(np.float64)
    vals = []
    desc = threads = None
    # every sample keeps every core busy (4 targets per core at least); the
    # whole run stays at about 2 * cpu_seconds plus the warm-up samples
    for _ in range(args.warmup):
        oracle_sample(prob, 0.0, K64=K64)
    for k in range(args.steps):
        v, desc, threads = oracle_sample(prob, 2 * args.cpu_seconds / max(args.steps, 1),
                                         seed=1 + k, K64=K64)
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
    """Device state and the step calls of one benchmark workload."""

    def __init__(self, sp, args, dev, seed):
        import numpy as np
        import torch
        self.sp, self.args, self.dev = sp, args, dev
        self.acc = {"kahan": sp.ACC_KAHAN32, "fp64": sp.ACC_FP64,
                    "fp64pair": sp.ACC_FP64_PAIR}[args.acc]
        if args.workload == "batched":
            import inputs
            self.probs = inputs.make_batched(seed=seed)[:max(1, args.trajectories)]
        else:
            self.probs = [load_problem(args.workload, seed, args.shot_stride)]
        self.batched = args.workload == "batched"
        self.one_launch = not args.two_launches
        self.off = [0]
        for p in self.probs:
            self.off.append(self.off[-1] + p.N)
        self.Ns = self.probs[0].Ns
        K = np.ascontiguousarray(np.concatenate([p.K for p in self.probs]))
        # pinned host copies: the inputs every step copies in, and the result
        # it copies back (the pattern evolves step by step, as in the method)
        self.Kh = torch.from_numpy(K).pin_memory()
        self.rhoh = [torch.from_numpy(p.grid.rho).pin_memory() for p in self.probs]
        self.K = self.Kh.to(dev)
        self.host_current = True        # Kh holds the latest pattern (else K on the device)
        self.rhos = [r.to(dev) for r in self.rhoh]
        self.grids = [sp.make_grid(r, p.grid.lo, p.grid.hi, p.grid.n)
                      for r, p in zip(self.rhos, self.probs)]
        self.hgrid = sp.make_grid(self.rhoh[0], self.probs[0].grid.lo, self.probs[0].grid.hi,
                                  self.probs[0].grid.n)
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
        self.kbytes = int(self.Kh.numel() * self.Kh.element_size())
        self.rhobytes = int(sum(r.numel() * r.element_size() for r in self.rhoh))

    def constraint_excess(self):
        """Largest constraint excess of the current pattern over all shots
        (eq. constraints): max |k[n+1]-k[n]| / alpha - 1, max
        |k[n+2]-2k[n+1]+k[n]| / beta - 1 and max |k|_inf - box; <= 0 where
        the pattern is feasible.  The steps run a fixed number of projection
        iterations, so small positive excesses are expected."""
        import numpy as np
        K = (self.Kh if self.host_current else self.K.cpu()).numpy().astype(np.float64)
        ea = eb = ex = -np.inf
        for b, p in enumerate(self.probs):
            S = K[self.off[b]:self.off[b + 1]].reshape(p.Nc, p.Ns, 3)
            if p.Ns > 1 and np.isfinite(p.proj.alpha):
                d1 = np.sqrt(((S[:, 1:] - S[:, :-1]) ** 2).sum(-1)).max()
                ea = max(ea, d1 / p.proj.alpha - 1.0)
            if p.Ns > 2 and np.isfinite(p.proj.beta):
                d2 = np.sqrt(((S[:, 2:] - 2.0 * S[:, 1:-1] + S[:, :-2]) ** 2).sum(-1)).max()
                eb = max(eb, d2 / p.proj.beta - 1.0)
            ex = max(ex, float(np.abs(S).max()) - p.proj.box)
        return {"alpha_rel": float(ea), "beta_rel": float(eb), "box": float(ex),
                "n_pit": int(self.probs[0].proj.n_iter),
                "note": "largest excess over all shots of the pattern after the timed steps "
                        "(<= 0: feasible); fixed-iteration projections"}

    def step_device(self):
        """One step on device-resident K (asynchronous)."""
        self.host_current = False
        sp = self.sp
        if self.batched:
            sp.sparkling_step_batched(self.ctx, self.K, self.off, self.Ns, self.grids, self.etas,
                                      self.projs, self.acc, graph=True,
                                      one_launch=self.one_launch)
        else:
            p = self.probs[0]
            sp.sparkling_step(self.ctx, self.K, p.Nc, p.Ns, self.grids[0], p.eta, self.projs[0],
                              self.acc)

    def step_host(self, stream):
        """One step from and to the pinned host buffers (blocking).  Returns
        the CUDA events around the device work when they are recorded here
        (the batched step), else None (the library's STEP scope times it)."""
        import torch
        sp = self.sp
        self.host_current = True
        if not self.batched:
            p = self.probs[0]
            sp.sparkling_step_host(self.ctx, self.Kh, p.Nc, p.Ns, self.hgrid, self.rhoh[0],
                                   p.eta, self.projs[0], self.acc)
            return None
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        self.K.copy_(self.Kh, non_blocking=True)
        for r, rh in zip(self.rhos, self.rhoh):
            r.copy_(rh, non_blocking=True)
        e0.record(stream)
        self.step_device()
        e1.record(stream)
        self.Kh.copy_(self.K, non_blocking=True)
        stream.synchronize()
        sp.sparkling_status(self.ctx)
        return e0, e1


def run_ours(args):
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
    sp.sparkling_set_step_path(ctx, args.path)
    sp.sparkling_set_projection(ctx, sp.PROJECTION_MIXED if args.projection == "mixed"
                                else sp.PROJECTION_FP64)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    field_build_ms = None
    mesh_build_ms = None
    fast = args.attraction == "field" or args.repulsion == "mesh"
    if args.attraction == "field":
        sp.sparkling_set_attraction(ctx, sp.ATTRACTION_FIELD)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        sp.sparkling_attraction_field(ctx, w.grids[0])      # blocking
        field_build_ms = (time.perf_counter() - t0) * 1e3
    if args.repulsion == "mesh":
        sp.sparkling_set_repulsion(ctx, sp.REPULSION_MESH,
                                   sp.make_mesh(args.mesh_cells, args.mesh_sigma, args.mesh_rc))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        w.step_device()                           # builds the kernel spectra (blocking)
        sp.sparkling_status(ctx)
        mesh_build_ms = (time.perf_counter() - t0) * 1e3

    # The fast modes keep the density's node field across steps, which a
    # host-buffer step (new density every call) would rebuild: they time the
    # device-resident step, and their e2e leg (optional) is a separate loop.
    # The exact paths run one loop of host-buffer steps for both numbers.
    one_loop = not fast

    def one_step(timed):
        flush.zero_()                        # evict L2 between steps (outside the timing)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        if one_loop:
            ev = w.step_host(stream)
        else:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            w.step_device()
            e1.record(stream)
            e1.synchronize()
            ev = (e0, e1)
        t1 = time.perf_counter()
        return (t1 - t0), ev

    for _ in range(args.warmup):
        one_step(False)
    sp.sparkling_status(ctx)
    torch.cuda.synchronize(dev)

    sp.sparkling_set_timing(ctx, True)
    sp.sparkling_kernel_times(ctx, reset=True)
    launches0 = sp.sparkling_launch_count(ctx)
    clocks = ClockSampler(local, args.clock_log)
    clocks.start()
    barrier()
    torch.cuda.synchronize(dev)
    wall_s, evs = [], []
    for _ in range(args.steps):
        dt, ev = one_step(True)
        wall_s.append(dt)
        if ev is not None:
            evs.append(ev)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    sp.sparkling_status(ctx)
    launches = sp.sparkling_launch_count(ctx) - launches0
    ktimes = sp.sparkling_kernel_times(ctx, reset=True)
    sp.sparkling_set_timing(ctx, False)

    # device time of the timed steps: the library's STEP scopes (single
    # trajectory) or the events around each batched step
    if evs:
        step_ms = [a.elapsed_time(b) for a, b in evs]
    else:
        ms, n = ktimes["step"]
        if n != args.steps:
            raise RuntimeError(f"expected {args.steps} timed step scopes, got {n}")
        step_ms = [ms / n] * n
    local_ms = sum(step_ms)
    total_ms = reduce_max(local_ms, dev)
    pairs_all = reduce_sum(float(w.pairs * args.steps), dev)
    value = pairs_all / (total_ms * 1e-3)

    e2e = None
    if one_loop:
        e2e_s = reduce_max(sum(wall_s), dev)
        e2e = {"value": pairs_all / e2e_s, "unit": "pairs/s",
               "h2d_bytes_per_step": w.kbytes + w.rhobytes, "d2h_bytes_per_step": w.kbytes,
               "seconds_per_step": e2e_s / args.steps,
               "note": "the same timed steps: each a sparkling_step_host call (pinned K and "
                       "density copied in, K copied back), wall clock around the call"}
    elif not args.no_e2e:
        # fast modes: the host-buffer step rebuilds the density's node field
        # every call (a new density arrives with each call)
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            w.step_host(stream)
        t1 = time.perf_counter()
        barrier()
        e2e_s = reduce_max(t1 - t0, dev)
        e2e = {"value": pairs_all / e2e_s, "unit": "pairs/s",
               "h2d_bytes_per_step": w.kbytes + w.rhobytes, "d2h_bytes_per_step": w.kbytes,
               "seconds_per_step": e2e_s / args.steps,
               "note": "separate loop of sparkling_step_host calls"}

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    probe = measure_probe() if rank == 0 else {}
    rsq = probe.get("rsqrt") if probe else None
    rate = float(round(rsq)) if rsq else float(SFU_RSQ_PER_SM_CLK)
    peak = sms * rate * max_mhz * 1e6
    if w.batched or ktimes["engine"][1]:
        # the engine (with the symmetric repulsion, as its items or in the
        # kernel ahead of it) takes one reciprocal square root per attraction
        # pair and one per unordered repulsion pair: N_b*P_b + N_b*(N_b-1)/2
        kname = "engine"
        kpairs = sum(p.N * int(p.grid.rho.size) + p.N * (p.N - 1) // 2 for p in w.probs)
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
    traffic = None
    if kname == "attraction" and not w.batched:
        traffic = attraction_traffic(w.probs[0], args)
    roof = {"bound": "alu", "achieved": achieved / 1e9 if achieved else None,
            "peak": peak / 1e9, "unit": "Gpair/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": traffic["bytes_per_launch"] if traffic else None,
            "kernel": kname,
            "peak_basis": f"{sms} SMs x {rate:g} MUFU.RSQ/clk/SM x {max_mhz:.0f} MHz max SM clock "
                          f"(one reciprocal square root per pair; probe measured "
                          f"{rsq if rsq else 'n/a'} RSQ/clk/SM)"}
    if kname == "engine":
        roof["unit"] = "G reciprocal square roots/s"
        roof["note"] = ("achieved counts the step's reciprocal square roots: one per attraction "
                        "pair and one per unordered repulsion pair (N_b*P_b + N_b*(N_b-1)/2)")
    if traffic:
        roof["traffic_basis"] = traffic["basis"]
    if clk and achieved:
        roof["frac_at_measured_clock"] = achieved / (sms * rate * clk["sm_mhz"] * 1e6)
    tot_k = max(sum(v[0] for k, v in ktimes.items() if k != "step"), 1e-9)
    kernels = {k: {"ms_total": round(ms, 3), "launches": n, "share": round(ms / tot_k, 4)}
               for k, (ms, n) in ktimes.items() if n and k != "step"}
    if not w.batched and ktimes["repulsion"][1] and args.repulsion == "direct":
        rep_ms, rep_n = ktimes["repulsion"]
        per = rep_ms / rep_n * 1e-3
        kernels["repulsion"]["gpair_per_s"] = w.N * (w.N - 1) / per / 1e9
        # FP32-pipe bound of the symmetric kernel: 12 FP32 lane operations per
        # unordered pair on 128 lanes per SM per clock
        kernels["repulsion"]["frac_of_fp32_bound"] = (
            w.N * (w.N - 1) / 2 / per / (sms * 128.0 / 12.0 * max_mhz * 1e6))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, desc, threads = oracle_sample(w.probs[0], args.cpu_seconds)
        cpu = {"value": v, "unit": "pairs/s", "cores": threads, "kind": "oracle", "sample": desc}

    if rank == 0:
        p0 = w.probs[0]
        proj_form = ("mixed FP32/FP64 projection" if args.projection == "mixed"
                     else "FP64 projection (duals, primal, step)")
        acc_form = {"kahan": "compensated-f32 per-target sums",
                    "fp64": "f64 per-target sums of f32 row sums",
                    "fp64pair": "every attraction pair term added in f64"}[args.acc]
        out = {
            "metric": "pair_interactions_per_s", "value": value, "unit": "pairs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": f"f32 pairs, {acc_form}, {proj_form}",
            "data": "synthetic",
            "config": {"workload": w.desc, "N": w.N, "P": int(p0.grid.rho.size),
                       "trajectories": len(w.probs), "Ns": w.Ns, "pairs_per_step": w.pairs,
                       "n_pit": p0.proj.n_iter,
                       "path": (("engine, one launch" if w.one_launch else "engine")
                                if w.batched else
                                "engine, one launch" if ktimes["engine"][1] else "kernels"),
                       "l2": "flushed (512 MB write) before every step", "acc": args.acc,
                       "projection": args.projection,
                       "attraction": args.attraction, "repulsion": args.repulsion,
                       "shapes": ("autotuned" if args.shape_attraction < 0
                                  and args.shape_repulsion < 0 else
                                  f"pinned: attraction {args.shape_attraction}, "
                                  f"repulsion {args.shape_repulsion} (-1: autotuned)")},
            "roofline": roof, "kernels": kernels, "clocks": clk, "e2e": e2e,
            "cpu_baseline": cpu, "gpu_launches": launches,
            "constraints": w.constraint_excess(),
            "seconds_per_iteration": total_ms / args.steps / 1e3,
            "step_ms": [round(v, 3) for v in step_ms],
            "autotuner": [l for l in sp.sparkling_tuning_report(ctx).splitlines() if l],
            "alu_probe_per_sm_clk": probe or None,
        }
        if mesh_build_ms is not None:
            out["mesh"] = {
                "cells": args.mesh_cells, "sigma_cells": args.mesh_sigma,
                "rc_sigmas": args.mesh_rc, "first_step_ms": mesh_build_ms,
                "note": "particle-particle particle-mesh repulsion; the first step (with the "
                        "tuner's trials) builds the kernel spectra once; value counts "
                        "N*P + N*(N-1) equivalent pairs"}
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
