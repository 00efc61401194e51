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
    ap.add_argument("--workload", choices=("hr", "diff", "medium", "small", "tiny"), default="hr")
    ap.add_argument("--acc", choices=("kahan", "fp64"), default="kahan")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target duration of the oracle sample")
    a = ap.parse_args(argv)
    if a.steps is None:
        a.steps = 1 if a.workload == "hr" else 3
    if a.warmup < 3:
        ap.error("--warmup must be >= 3")
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

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{index}.csv")

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


def measure_rsq_rate():
    """Run alu_peak_probe.cu (built with nvcc) and return the measured
    MUFU.RSQ results per SM per clock, or None when it cannot run."""
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
            return None
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    m = re.search(r"^rsqrt\s+ops/SM/clk = ([0-9.]+)", r.stdout, re.M)
    return float(m.group(1)) if m else None


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
    prob = load_problem(args.workload, 0)
    N, P = prob.N, int(prob.grid.rho.size)
    vals = []
    desc = threads = None
    for _ in range(args.warmup):
        oracle_sample(prob, min(args.cpu_seconds, 3.0) / 3)
    for _ in range(args.steps):
        v, desc, threads = oracle_sample(prob, args.cpu_seconds / max(args.steps, 1))
        vals.append(v)
    value = statistics.median(vals)
    unit = "pairs/s"
    step_s = pairs_per_step(N, P) / value
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

    prob = load_problem(args.workload, seed=rank)
    N, P = prob.N, int(prob.grid.rho.size)
    acc = sp.ACC_KAHAN32 if args.acc == "kahan" else sp.ACC_FP64
    K0 = torch.from_numpy(prob.K).to(dev)
    K = K0.clone()
    rho = torch.from_numpy(prob.grid.rho).to(dev)
    grid = sp.make_grid(rho, prob.grid.lo, prob.grid.hi, prob.grid.n)
    pp = prob.proj
    proj = sp.make_proj(pp.alpha, pp.beta, pp.box, pp.n_iter, pp.pin_index, pp.pin)
    ctx = sp.sparkling_create(local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        sp.sparkling_step(ctx, K, prob.Nc, prob.Ns, grid, prob.eta, proj, acc)
    sp.sparkling_status(ctx)
    torch.cuda.synchronize(dev)

    sp.sparkling_set_timing(ctx, True)
    sp.sparkling_kernel_times(ctx, reset=True)
    launches0 = sp.sparkling_launch_count(ctx)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize(dev)
    step_ms = []
    for _ in range(args.steps):
        flush.zero_()                        # evict L2 between timed steps (not timed)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sp.sparkling_step(ctx, K, prob.Nc, prob.Ns, grid, prob.eta, proj, acc)
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
    pairs_all = reduce_sum(float(pairs_per_step(N, P) * args.steps), dev)
    value = pairs_all / (total_ms * 1e-3)

    # dominant kernel: the attraction sum (N*P pairs per launch)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    import json as _json
    peaks = {}
    try:
        peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    att_ms, att_n = ktimes["attraction"]
    rep_ms, rep_n = ktimes["repulsion"]
    att_pairs = N * P
    achieved = att_pairs / (att_ms / att_n * 1e-3) if att_n else None
    rsq = measure_rsq_rate() if rank == 0 else None
    rate = float(round(rsq)) if rsq else float(SFU_RSQ_PER_SM_CLK)
    peak = sms * rate * max_mhz * 1e6
    roof = {"bound": "alu", "achieved": achieved / 1e9 if achieved else None,
            "peak": peak / 1e9, "unit": "Gpair/s",
            "frac": (achieved / peak) if achieved else None, "traffic": None,
            "kernel": "attraction",
            "peak_basis": f"{sms} SMs x {rate:g} MUFU.RSQ/clk/SM x {max_mhz:.0f} MHz max SM clock "
                          f"(one reciprocal square root per pair; probe measured "
                          f"{rsq if rsq else 'n/a'} RSQ/clk/SM)"}
    if clk and achieved:
        roof["frac_at_measured_clock"] = achieved / (sms * rate * clk["sm_mhz"] * 1e6)
    kernels = {k: {"ms_total": round(ms, 3), "launches": n,
                   "share": round(ms / max(sum(v[0] for v in ktimes.values()), 1e-9), 4)}
               for k, (ms, n) in ktimes.items()}
    if rep_n:
        kernels["repulsion"]["gpair_per_s"] = N * (N - 1) / (rep_ms / rep_n * 1e-3) / 1e9

    e2e = None
    if not args.no_e2e:
        Kh = torch.from_numpy(prob.K).pin_memory()
        rhoh = torch.from_numpy(prob.grid.rho).pin_memory()
        hgrid = sp.make_grid(rhoh, prob.grid.lo, prob.grid.hi, prob.grid.n)
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sp.sparkling_step_host(ctx, Kh, prob.Nc, prob.Ns, hgrid, rhoh, prob.eta, proj, acc)
        t1 = time.perf_counter()
        barrier()
        e2e_s = reduce_max(t1 - t0, dev)
        e2e = {"value": pairs_all / e2e_s, "unit": "pairs/s",
               "h2d_bytes_per_step": int(Kh.numel() * Kh.element_size() + rhoh.numel() * 4),
               "d2h_bytes_per_step": int(Kh.numel() * Kh.element_size())}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, desc, threads = oracle_sample(prob, args.cpu_seconds)
        cpu = {"value": v, "unit": "pairs/s", "cores": threads, "kind": "oracle", "sample": desc}

    if rank == 0:
        out = {
            "metric": "pair_interactions_per_s", "value": value, "unit": "pairs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 pairs, " + ("compensated-f32" if acc == 0 else "f64")
            + " per-target sums, f64 projection",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {prob.recipe}", "N": N, "P": P,
                       "Nc": prob.Nc, "Ns": prob.Ns, "pairs_per_step": pairs_per_step(N, P),
                       "n_pit": pp.n_iter, "l2": "flushed (512 MB write) between timed steps",
                       "acc": args.acc},
            "roofline": roof, "kernels": kernels, "clocks": clk, "e2e": e2e,
            "cpu_baseline": cpu, "gpu_launches": launches,
            "seconds_per_iteration": total_ms / args.steps / 1e3,
        }
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
