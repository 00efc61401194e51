"""Host-side logic of bench.py on the CPU: argument defaults, the pair
count, the max/sum-over-ranks timing reductions with two gloo ranks, and the
reference arm (the FP64 oracle timed on the host cores) on a tiny workload."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_defaults_and_pair_count():
    a = bench.parse_args([])
    assert (a.gpus, a.workload, a.warmup, a.steps, a.impl) == (1, "hr", 3, 1, "ours")
    with pytest.raises(SystemExit):
        bench.parse_args(["--warmup", "2"])
    assert bench.pairs_per_step(10, 7) == 10 * 7 + 10 * 9


def test_constraint_excess_of_the_pattern():
    """The bench line's constraint report: a straight constant-speed shot at
    exactly the amplitude bound has excess 0 in alpha and -1 in beta (no
    second differences), and doubling its speed makes the alpha excess 1;
    samples beyond the box show as a positive box excess."""
    import types
    import numpy as np
    import torch
    import inputs
    Ns, a, b, box = 8, 0.01, 0.001, 0.5
    shot = np.zeros((Ns, 3))
    shot[:, 0] = np.arange(Ns) * a - 0.03
    probs = [types.SimpleNamespace(N=Ns, Nc=1, Ns=Ns, proj=inputs.Proj(a, b, box))]
    w = types.SimpleNamespace(probs=probs, off=[0, Ns], host_current=True,
                              Kh=torch.from_numpy(shot), K=None)
    r = bench.Workload.constraint_excess(w)
    assert abs(r["alpha_rel"]) < 1e-12 and r["beta_rel"] == pytest.approx(-1.0)
    assert r["box"] == pytest.approx(max(abs(shot.min()), shot.max()) - box)
    w.Kh = torch.from_numpy(2.0 * shot + np.array([0.0, 0.0, 0.6]))
    r = bench.Workload.constraint_excess(w)
    assert r["alpha_rel"] == pytest.approx(1.0) and r["box"] == pytest.approx(0.1)


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mx = bench.reduce_max(float(rank + 1))
    sm = bench.reduce_sum(float(10 * (rank + 1)))
    bench.barrier()
    out.put((rank, mx, sm))
    dist.destroy_process_group()


def test_two_rank_reductions_with_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2.0, 30.0), (1, 2.0, 30.0)]


def test_reference_arm_prints_one_line_on_rank0_only():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
           "tiny", "--steps", "1", "--warmup", "3", "--cpu-seconds", "0.2"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_traffic_figure_only_for_the_kernel_it_was_measured_on(tmp_path, monkeypatch):
    """The bench line's DRAM traffic comes from the committed ncu summary's
    fit, only for the density it was measured on and only while the
    attraction kernel's source hashes to the value recorded there."""
    import inputs
    a = bench.parse_args([])
    p = inputs.make_problem("tiny")
    prof = tmp_path / "traffic.md"
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(prof))
    assert bench.attraction_traffic(p, a) is None                 # no summary
    sha = bench.attraction_source_sha()
    P = int(p.grid.rho.size)
    prof.write_text(f"traffic-fit: kernel_sha={sha} density={P} bytes_const=1.5e6 "
                    f"bytes_per_target=100\n")
    t = bench.attraction_traffic(p, a)
    assert t["bytes_per_launch"] == pytest.approx(1.5e6 + 100 * p.N)
    prof.write_text(f"traffic-fit: kernel_sha=0000000000000000 density={P} bytes_const=1.5e6 "
                    f"bytes_per_target=100\n")
    assert bench.attraction_traffic(p, a) is None                 # another kernel source
    prof.write_text(f"traffic-fit: kernel_sha={sha} density={P + 1} bytes_const=1.5e6 "
                    f"bytes_per_target=100\n")
    assert bench.attraction_traffic(p, a) is None                 # another density
    assert bench.attraction_traffic(p, bench.parse_args(["--acc", "fp64pair"])) is None


def test_shot_stride_keeps_every_sth_shot():
    full = bench.load_problem("tiny", 0)
    sub = bench.load_problem("tiny", 0, 4)
    assert sub.Nc == (full.Nc + 3) // 4 and sub.Ns == full.Ns
    K = full.K.reshape(full.Nc, full.Ns, 3)[::4].reshape(-1, 3)
    assert (sub.K == K).all() and sub.eta == pytest.approx(1.0 / sub.N)
