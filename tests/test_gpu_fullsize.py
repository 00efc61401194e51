"""Parity at the full sizes of the synthetic workloads, through the same
C-ABI calls and launch configuration the benchmark uses.  The oracle computes
sampled targets / shots one by one; properties that hold at any size (zero
net repulsion, feasibility of the projection) cover the rest."""
import numpy as np
import pytest

import inputs
import oracle
from gpu_util import assert_grad_close, proj_tol_f32, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_02991_gb300 import build
    build.build()
    import paper_2108_02991_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(sp):
    c = sp.sparkling_create(0)
    yield c
    c.close()


def sample_targets(N, m, seed):
    return np.sort(np.random.default_rng(seed).choice(N, size=m, replace=False))


def test_medium_ten_iterations(sp, ctx):
    """512 x 512 spokes, 128^3 density, 10 projected-gradient steps with step
    1/N.  Each GPU iterate is fed to the oracle: the gradient on sampled
    targets at the first and last iteration, and the projection of every shot
    (K_t - eta G_t) at every iteration."""
    p = inputs.make_problem("medium")
    K = torch.from_numpy(p.K).cuda()
    rho = torch.from_numpy(p.grid.rho).cuda()
    g = sp.make_grid(rho, p.grid.lo, p.grid.hi, p.grid.n)
    pp = p.proj
    proj = sp.make_proj(pp.alpha, pp.beta, pp.box, pp.n_iter, pp.pin_index, pp.pin)
    idx = sample_targets(p.N, 128, 1)
    for it in range(p.iterations):
        Kt = K.cpu().numpy().astype(np.float64)
        G = sp.sparkling_grad(ctx, K, g, G=torch.empty(p.N, 3, dtype=torch.float64, device="cuda"))
        sp.sparkling_status(ctx)
        Gt = G.cpu().numpy()
        if it in (0, p.iterations - 1):
            _, _, G0 = oracle.forces(Kt, p.grid, targets=idx)
            assert_grad_close(Gt[idx], G0, f"G (iteration {it})")
        sp.sparkling_step(ctx, K, p.Nc, p.Ns, g, p.eta, proj)
        sp.sparkling_status(ctx)
        half = Kt - p.eta * Gt
        ref = oracle.project(half, p.Nc, p.Ns, pp.alpha, pp.beta, pp.box,
                             pp.pin_index, pp.pin, pp.n_iter)
        out = K.cpu().numpy()
        d = np.abs(out.astype(np.float64) - ref.astype(np.float32).astype(np.float64)).max()
        tol = proj_tol_f32(ref, half)
        assert d <= tol, f"iteration {it}: projection differs by {d:.2e} > {tol:.2e}"
        np.testing.assert_array_equal(out[:, :][pp.pin_index::p.Ns], 0.0)   # TE pin


def test_diff_autograd_backward_and_finite_differences(sp, ctx):
    """N = 1,048,576, 192^3 density, FP64 per-target accumulation: the energy
    is the forward of SparklingEnergy and its backward is the gradient kernel.
    The backward matches the oracle's G/N on 256 sampled targets and the
    central differences (h = 1e-4, FP64) of the terms of F that involve the
    perturbed sample (computed by the oracle) on 16 targets."""
    from paper_2108_02991_gb300 import sparkling_energy_fn
    p = inputs.make_problem("diff")
    N = p.N
    K = torch.from_numpy(p.K).cuda().requires_grad_(True)
    rho = torch.from_numpy(p.grid.rho).cuda()
    F = sparkling_energy_fn(K, rho, ctx, p.grid.lo, p.grid.hi, acc=sp.ACC_FP64)
    F.backward()
    dK = K.grad.double().cpu().numpy()
    K64 = p.K.astype(np.float64)
    idx = sample_targets(N, 256, 2)
    _, _, G0 = oracle.forces(K64, p.grid, targets=idx)
    assert_grad_close(dK[idx] * N, G0, "N * dF/dK")
    assert np.isfinite(float(F.detach()))

    h = 1e-4
    rng = np.random.default_rng(3)
    fd_idx = rng.choice(N, size=16, replace=False)
    fd, gp = [], []
    for i in fd_idx:
        c = int(rng.integers(3))
        vals = []
        for sgn in (1.0, -1.0):
            Kp = K64.copy()
            Kp[i, c] += sgn * h
            _, _, _, ea, er = oracle.forces(Kp, p.grid, targets=[i], energies=True)
            # terms of F that contain K_i: (1/N) ea_i - (1/N^2) er_i
            vals.append(ea[0] / N - er[0] / (N * N))
        fd.append((vals[0] - vals[1]) / (2 * h) * N)
        gp.append(dK[i, c] * N)
    assert_grad_close(np.array(gp), np.array(fd), "backward vs central differences")


def test_hr_sampled_targets_and_shots(sp, ctx):
    """4096 x 2560 samples, 256^3 density (2.9e14 pairs): the gradient in the
    benchmark's launch configuration on 64 sampled targets, zero net
    repulsion, and the projection of 8 sampled shots of K - eta G."""
    p = inputs.make_problem("hr")
    N = p.N
    K = torch.from_numpy(p.K).cuda()
    rho = torch.from_numpy(p.grid.rho).cuda()
    g = sp.make_grid(rho, p.grid.lo, p.grid.hi, p.grid.n)
    G = torch.empty(N, 3, dtype=torch.float64, device="cuda")
    R = torch.empty_like(G)
    sp.sparkling_grad(ctx, K, g, sp.ACC_KAHAN32, G=G, R=R)
    sp.sparkling_status(ctx)
    idx = sample_targets(N, 64, 4)
    K64 = p.K.astype(np.float64)
    A0, R0, G0 = oracle.forces(K64, p.grid, targets=idx)
    Gh = G.cpu().numpy()
    assert_grad_close(Gh[idx], G0, "G (HR)")
    assert_grad_close(R.cpu().numpy()[idx], R0, "R (HR)")
    net = R.sum(dim=0).abs().max().item() / R.abs().sum().item()
    assert net < 1e-6, f"net repulsion {net:.2e}"

    pp = p.proj
    half = torch.from_numpy(K64 - p.eta * Gh).cuda()
    proj = sp.make_proj(pp.alpha, pp.beta, pp.box, pp.n_iter, pp.pin_index, pp.pin)
    sp.sparkling_project(ctx, half, p.Nc, p.Ns, proj)
    sp.sparkling_status(ctx)
    shots = sample_targets(p.Nc, 8, 5)
    out = half.cpu().numpy()
    src = K64 - p.eta * Gh
    for c in shots:
        sl = slice(c * p.Ns, (c + 1) * p.Ns)
        ref = oracle.project(src[sl], 1, p.Ns, pp.alpha, pp.beta, pp.box, pp.pin_index, pp.pin,
                             pp.n_iter)
        np.testing.assert_allclose(out[sl], ref, rtol=0, atol=1e-11)
