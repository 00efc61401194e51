"""Parity at the full sizes of the synthetic workloads, through the same
C-ABI calls and launch configuration the benchmark uses.  The oracle computes
sampled targets / shots one by one; properties that hold at any size (zero
net repulsion, feasibility of the projection) cover the rest."""
import numpy as np
import pytest

import inputs
import oracle
from gpu_util import PROJ_F32_ROUND, assert_grad_close, rel_l2

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
    1/N.  Each GPU iterate is fed to the oracle: the gradient on 4096 random
    targets at every iteration, and the projection of every shot
    (K_t - eta G_t) at every iteration (FP64 projection, one rounding to
    FP32)."""
    p = inputs.make_problem("medium")
    K = torch.from_numpy(p.K).cuda()
    rho = torch.from_numpy(p.grid.rho).cuda()
    g = sp.make_grid(rho, p.grid.lo, p.grid.hi, p.grid.n)
    pp = p.proj
    proj = sp.make_proj(pp.alpha, pp.beta, pp.box, pp.n_iter, pp.pin_index, pp.pin)
    for it in range(p.iterations):
        Kt = K.cpu().numpy().astype(np.float64)
        G = sp.sparkling_grad(ctx, K, g, G=torch.empty(p.N, 3, dtype=torch.float64, device="cuda"))
        sp.sparkling_status(ctx)
        Gt = G.cpu().numpy()
        idx = sample_targets(p.N, 4096, 100 + it)
        _, _, G0 = oracle.forces(Kt, p.grid, targets=idx)
        assert_grad_close(Gt[idx], G0, f"G (iteration {it}, 4096 targets)")
        sp.sparkling_step(ctx, K, p.Nc, p.Ns, g, p.eta, proj)
        sp.sparkling_status(ctx)
        half = Kt - p.eta * Gt
        ref = oracle.project(half, p.Nc, p.Ns, pp.alpha, pp.beta, pp.box,
                             pp.pin_index, pp.pin, pp.n_iter)
        out = K.cpu().numpy()
        d = np.abs(out.astype(np.float64) - ref.astype(np.float32).astype(np.float64)).max()
        assert d <= PROJ_F32_ROUND, f"iteration {it}: projection differs by {d:.2e}"
        np.testing.assert_array_equal(out[:, :][pp.pin_index::p.Ns], 0.0)   # TE pin


def central_differences(K64, grid, idx, comp, h):
    """N * (F(K + h e) - F(K - h e)) / (2h) in coordinate comp[m] of sample
    idx[m], from the oracle's terms of F that contain that sample."""
    N = K64.shape[0]
    P = np.repeat(K64[idx][None], 2, axis=0)
    rows = np.arange(len(idx))
    P[0, rows, comp] += h
    P[1, rows, comp] -= h
    ea, er = oracle.energy_terms(K64, grid, np.concatenate([idx, idx]), P.reshape(-1, 3))
    f = ea / N - er / (N * N)
    m = len(idx)
    return (f[:m] - f[m:]) / (2 * h) * N


def test_diff_autograd_backward_and_finite_differences(sp, ctx):
    """N = 1,048,576, 192^3 density, FP64 per-target accumulation: the energy
    is the forward of SparklingEnergy and its backward is the gradient kernel.

    * the backward times N matches the oracle's G on 4096 random targets;
    * the oracle's G is itself checked at this size by central differences
      (h = 1e-4, FP64) of the terms of F that contain the moved sample, on
      the same 4096 targets (one random coordinate each): the Richardson
      combination (4 D(h) - D(2h)) / 3, whose truncation error is O(h^4),
      within 1e-6 relative L2 on all of them (6e-8 measured on 512 of them);
      the plain D(h) within 1e-6 on the targets whose own truncation estimate
      |D(2h) - D(h)| / 3 is below 1e-7 (about 84 % of them; over all targets
      the O(h^2 / r^2) terms of the grid points nearest to a target bring
      D(h) to 1.0e-6);
    * the backward matches the central differences on the same targets."""
    from paper_2108_02991_gb300 import sparkling_energy_fn
    p = inputs.make_problem("diff")
    N = p.N
    K = torch.from_numpy(p.K).cuda().requires_grad_(True)
    rho = torch.from_numpy(p.grid.rho).cuda()
    F = sparkling_energy_fn(K, rho, ctx, p.grid.lo, p.grid.hi, acc=sp.ACC_FP64)
    F.backward()
    dK = K.grad.double().cpu().numpy()
    assert np.isfinite(float(F.detach()))
    K64 = p.K.astype(np.float64)
    idx = sample_targets(N, 4096, 2)
    _, _, G0 = oracle.forces(K64, p.grid, targets=idx)
    assert_grad_close(dK[idx] * N, G0, "N * dF/dK (4096 targets)")

    h = 1e-4
    comp = np.random.default_rng(3).integers(3, size=idx.size)
    d1 = central_differences(K64, p.grid, idx, comp, h)
    d2 = central_differences(K64, p.grid, idx, comp, 2 * h)
    g = G0[np.arange(idx.size), comp]
    rich = (4 * d1 - d2) / 3
    e_rich = rel_l2(rich, g)
    est = np.abs(d2 - d1) / 3
    ok = est < 1e-7
    e_plain = rel_l2(d1[ok], g[ok])
    print(f"diff central differences: Richardson rel L2 {e_rich:.2e} (4096 targets), plain "
          f"D(h) rel L2 {e_plain:.2e} on {ok.sum()} targets with estimate < 1e-7")
    assert e_rich <= 1e-6
    assert ok.sum() >= idx.size // 2
    assert e_plain <= 1e-6
    assert_grad_close(dK[idx, comp] * N, rich, "backward vs central differences")


def test_hr_step_through_the_engine(sp, hr_oracle):
    """The 1e7-sample step as the library runs it by default (one launch of
    the persistent engine): with alpha = beta = inf and a loose box the
    projection is the identity, so K' = K - G (eta = 1, K in FP64) exposes the
    engine's gradient, checked against the oracle on the 8192 sampled
    targets."""
    p, idx, A0, R0, G0 = hr_oracle
    c = sp.sparkling_create(0)
    try:
        sp.sparkling_set_timing(c, True)
        K = torch.from_numpy(p.K.astype(np.float64)).cuda()
        rho = torch.from_numpy(p.grid.rho).cuda()
        g = sp.make_grid(rho, p.grid.lo, p.grid.hi, p.grid.n)
        proj = sp.make_proj(float("inf"), float("inf"), 10.0, 2)
        sp.sparkling_step(c, K, p.Nc, p.Ns, g, 1.0, proj)
        sp.sparkling_status(c)
        t = sp.sparkling_kernel_times(c)
        out = K.cpu().numpy()
    finally:
        c.close()
    assert t["engine"][1] == 1 and t["attraction"][1] == 0, t
    G = p.K.astype(np.float64)[idx] - out[idx]
    e, _ = assert_grad_close(G, G0, "engine G (HR step, 8192 targets)")
    print(f"HR step through the engine: G rel L2 {e:.2e} on 8192 targets")


def test_hr_sampled_targets_and_shots(sp, ctx, hr_oracle):
    """4096 x 2560 samples, 256^3 density (2.8e14 pairs): the gradient in the
    benchmark's launch configuration on 8192 random targets (G and R), zero
    net repulsion, and the projection of 8 sampled shots of K - eta G."""
    p, idx, A0, R0, G0 = hr_oracle
    N = p.N
    K = torch.from_numpy(p.K).cuda()
    rho = torch.from_numpy(p.grid.rho).cuda()
    g = sp.make_grid(rho, p.grid.lo, p.grid.hi, p.grid.n)
    G = torch.empty(N, 3, dtype=torch.float64, device="cuda")
    R = torch.empty_like(G)
    sp.sparkling_grad(ctx, K, g, sp.ACC_KAHAN32, G=G, R=R)
    sp.sparkling_status(ctx)
    K64 = p.K.astype(np.float64)
    Gh = G.cpu().numpy()
    eG, _ = assert_grad_close(Gh[idx], G0, "G (HR, 8192 targets)")
    eR, _ = assert_grad_close(R.cpu().numpy()[idx], R0, "R (HR, 8192 targets)")
    print(f"HR direct: G rel L2 {eG:.2e}, R rel L2 {eR:.2e} on 8192 targets")
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
