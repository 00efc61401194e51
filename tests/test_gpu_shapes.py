"""Every tile shape of the pair kernels, pinned with sparkling_set_shape,
against the FP64 oracle.

* the three attraction shapes (128 / 256 / 512 threads) and the four shapes
  of the symmetric repulsion (256 threads: 2 sources per lane with the
  targets paired in the 64-bit registers, 4 sources per lane, 2 sources per
  lane with the sources paired; 128 threads with 8 targets per lane and the
  sources paired), on 7,703 samples (8 target tiles, the last ragged) and a
  random density whose rows are not a multiple of 4: A, R, G and the energy,
  plain and regularised kernel;
* the two-launch batched step (batched symmetric kernel + engine) with each
  repulsion shape: the gradient recovered from an unconstrained step.
"""
import numpy as np
import pytest

import inputs
import oracle
from gpu_util import assert_grad_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
INF = float("inf")

SHAPES = [("attraction", v) for v in range(3)] + [("repulsion", v) for v in range(4)]


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_02991_gb300 import build
    build.build()
    import paper_2108_02991_gb300 as m
    return m


def random_grid(nx, ny, nz, seed):
    rho = np.random.default_rng(seed).uniform(0.0, 1.0, size=(nz, ny, nx))
    return inputs.Grid((nx, ny, nz), -0.5, 0.5, (rho / rho.sum()).astype(np.float32))


@pytest.fixture(scope="module")
def problem():
    K = inputs.radial_spokes(11, 700, 0.23, jitter=1e-3, seed=81, dtype=np.float32)
    extra = np.array([[0.3, -0.2, 0.1], [0.3, -0.2, 0.1], [-0.41, 0.02, 0.37]], np.float32)
    return np.concatenate([K, extra]), random_grid(29, 31, 17, 82)   # a coincident pair


@pytest.mark.parametrize("eps", [0.0, 0.01])
@pytest.mark.parametrize("kernel,variant", SHAPES)
def test_pinned_shape_matches_oracle(sp, problem, kernel, variant, eps):
    K, grid = problem
    K64 = K.astype(np.float64)
    c = sp.sparkling_create(0)
    try:
        sp.sparkling_set_shape(c, kernel, variant)
        if eps:
            sp.sparkling_set_regularisation(c, eps)
        Kd = torch.from_numpy(K).cuda()
        g = sp.make_grid(torch.from_numpy(grid.rho).cuda(), grid.lo, grid.hi, grid.n)
        G = torch.empty(K.shape, dtype=torch.float64, device="cuda")
        A = torch.empty_like(G)
        R = torch.empty_like(G)
        sp.sparkling_grad(c, Kd, g, sp.ACC_KAHAN32, G=G, A=A, R=R)
        sp.sparkling_status(c)
        F, Fa, Fr = sp.sparkling_energy(c, Kd, g, sp.ACC_KAHAN32)
        report = sp.sparkling_tuning_report(c)
    finally:
        c.close()
    # the pinned kernel was not tuned (no trial lines of it in the report)
    trials = [l for l in report.splitlines() if l.endswith("pairs/s")]
    prefix = "attraction gxp" if kernel == "attraction" else "repulsion symmetric"
    assert not [l for l in trials if l.startswith(prefix)], report
    A0, R0, G0 = oracle.forces(K64, grid, eps=eps)
    assert_grad_close(A.cpu().numpy(), A0, f"A ({kernel} shape {variant})")
    assert_grad_close(R.cpu().numpy(), R0, f"R ({kernel} shape {variant})")
    cond = (np.linalg.norm(A0) + np.linalg.norm(R0)) / np.linalg.norm(G0) / 2
    assert_grad_close(G.cpu().numpy(), G0, f"G ({kernel} shape {variant})",
                      rel=1e-5 * max(cond, 1.0))
    _, Fa0, Fr0 = oracle.energy(K64, grid, eps=eps)
    assert Fa == pytest.approx(Fa0, rel=1e-6)
    assert Fr == pytest.approx(Fr0, rel=1e-6)


@pytest.mark.parametrize("variant", range(4))
def test_batched_step_with_each_repulsion_shape(sp, variant):
    """alpha = beta = inf and a loose box make the projection the identity,
    so G = (K - K') / eta exposes the batched kernels' gradient."""
    Ns = 128
    shots = [9, 2, 17]
    rng = np.random.default_rng(83)
    Ks, grids = [], []
    for b, nc in enumerate(shots):
        Kb = np.cumsum(rng.normal(scale=3e-3, size=(nc, Ns, 3)), axis=1).reshape(-1, 3)
        Ks.append(np.clip(Kb + rng.uniform(-0.2, 0.2, size=(1, 3)), -0.45, 0.45))
        grids.append(random_grid(*[(20, 10, 8), (7, 7, 7), (32, 8, 4)][b], seed=84 + b))
    etas = [1.0, 0.5, 2.0]
    off = np.concatenate([[0], np.cumsum([k.shape[0] for k in Ks])])
    c = sp.sparkling_create(0)
    try:
        sp.sparkling_set_shape(c, "repulsion", variant)
        K = torch.from_numpy(np.concatenate(Ks)).cuda()
        rhos = [torch.from_numpy(g.rho).cuda() for g in grids]
        gs = [sp.make_grid(r, g.lo, g.hi, g.n) for r, g in zip(rhos, grids)]
        ps = [sp.make_proj(INF, INF, 10.0, 3) for _ in grids]
        sp.sparkling_step_batched(c, K, off, Ns, gs, etas, ps, graph=False, one_launch=False)
        sp.sparkling_status(c)
        out = K.cpu().numpy()
    finally:
        c.close()
    for b in range(len(Ks)):
        G = (Ks[b] - out[off[b]:off[b + 1]]) / etas[b]
        _, _, G0 = oracle.forces(Ks[b], grids[b])
        assert_grad_close(G, G0, f"batched G of trajectory {b} (repulsion shape {variant})")
