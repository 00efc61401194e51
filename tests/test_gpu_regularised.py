"""Regularised kernel H(r) = sqrt(r^2 + eps^2) (Sec. II-C, choice of step
size) through the C ABI against the oracle with the same eps: gradient and
energy on ragged sizes with coincident samples and samples on grid points,
the batched engine (the gradient it applies, recovered from an
unconstrained step, and graph replay after eps changes), and the node field
of the fast attraction."""
import numpy as np
import pytest

import inputs
import oracle
from gpu_util import assert_grad_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
INF = float("inf")


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_02991_gb300 import build
    build.build()
    import paper_2108_02991_gb300 as m
    return m


def random_grid(nx, ny, nz, seed, lo=-0.5, hi=0.5):
    rho = np.random.default_rng(seed).uniform(0.0, 1.0, size=(nz, ny, nx))
    rho = (rho / rho.sum()).astype(np.float32)
    return inputs.Grid((nx, ny, nz), lo, hi, rho)


def samples(N, seed, grid):
    """Uniform samples with a few exact duplicates and a few samples placed
    on grid points (positions exactly representable in float32)."""
    rng = np.random.default_rng(seed)
    K = rng.uniform(-0.48, 0.48, size=(N, 3)).astype(np.float32)
    K[1] = K[0]
    K[N // 2] = K[N // 3]
    nx, ny, nz = grid.n
    for m in range(5):
        q = [int(rng.integers(n)) for n in (nx, ny, nz)]
        K[5 + m] = [grid.lo + (q[a] + 0.5) * (grid.hi - grid.lo) / grid.n[a] for a in range(3)]
    return K


@pytest.mark.parametrize("eps,acc", [(0.02, 0), (0.02, 1), (1e-3, 0), (0.3, 0)])
def test_grad_and_energy_regularised(sp, eps, acc):
    grid = random_grid(16, 8, 8, seed=41)        # dyadic cells: grid points exact in float
    N = 2 * 1024 + 77                            # three target tiles, ragged
    K = samples(N, 42, grid)
    ctx = sp.sparkling_create(0)
    try:
        sp.sparkling_set_regularisation(ctx, eps)
        Kd = torch.from_numpy(K).cuda()
        rho = torch.from_numpy(grid.rho).cuda()
        g = sp.make_grid(rho, grid.lo, grid.hi, grid.n)
        G = torch.empty(N, 3, dtype=torch.float64, device="cuda")
        A = torch.empty_like(G)
        R = torch.empty_like(G)
        sp.sparkling_grad(ctx, Kd, g, acc, G=G, A=A, R=R)
        sp.sparkling_status(ctx)
        A0, R0, G0 = oracle.forces(K.astype(np.float64), grid, eps=eps)
        assert_grad_close(R.cpu().numpy(), R0, f"R (eps {eps})")
        assert_grad_close(A.cpu().numpy(), A0, f"A (eps {eps})")
        # G = A - R: an eps far above the sample spacing (0.3) flattens both
        # terms until they cancel to 1/40 of their size, and the subtraction's
        # condition number (|A| + |R|) / (2 |G|) scales the relative gate there
        cond = (np.linalg.norm(A0) + np.linalg.norm(R0)) / np.linalg.norm(G0) / 2
        rel = 1e-5 if eps < 0.1 else 1e-5 * cond
        assert_grad_close(G.cpu().numpy(), G0, f"G (eps {eps}, condition {cond:.1f})", rel=rel)
        F, Fa, Fr = sp.sparkling_energy(ctx, Kd, g, acc)
        F0, Fa0, Fr0 = oracle.energy(K.astype(np.float64), grid, eps=eps)
        assert Fa == pytest.approx(Fa0, rel=1e-6)
        assert Fr == pytest.approx(Fr0, rel=1e-6)
        assert F == pytest.approx(F0, abs=1e-6 * (Fa0 + Fr0))
        # back to the plain norm on the same context
        sp.sparkling_set_regularisation(ctx, 0.0)
        sp.sparkling_grad(ctx, Kd, g, acc, G=G)
        sp.sparkling_status(ctx)
        _, _, Gp = oracle.forces(K.astype(np.float64), grid)
        assert_grad_close(G.cpu().numpy(), Gp, "G (eps back to 0)")
    finally:
        ctx.close()


def test_batched_engine_regularised_and_graph_recapture(sp):
    """The engine applies the regularised gradient (alpha = beta = inf, loose
    box: K' = K - eta G); a graph captured with one eps is not replayed
    after eps changes."""
    Ns = 128
    rng = np.random.default_rng(43)
    shots = [5, 9]
    grids = [random_grid(12, 10, 8, seed=44), random_grid(8, 8, 8, seed=45)]
    Ks = [rng.uniform(-0.45, 0.45, size=(nc * Ns, 3)) for nc in shots]
    off = np.concatenate([[0], np.cumsum([k.shape[0] for k in Ks])])
    rhos = [torch.from_numpy(g.rho).cuda() for g in grids]
    gs = [sp.make_grid(r, g.lo, g.hi, g.n) for r, g in zip(rhos, grids)]
    ps = [sp.make_proj(INF, INF, 10.0, 3) for _ in Ks]
    etas = [1.0, 1.0]
    ctx = sp.sparkling_create(0)
    try:
        K0 = torch.from_numpy(np.concatenate(Ks)).cuda()
        K = torch.empty_like(K0)                  # one buffer: the graph key stays the same
        for eps in (0.05, 0.05, 0.05, 0.01):      # eager, capture, replay, new eps
            sp.sparkling_set_regularisation(ctx, eps)
            K.copy_(K0)
            sp.sparkling_step_batched(ctx, K, off, Ns, gs, etas, ps, graph=True)
            sp.sparkling_status(ctx)
            out = K.cpu().numpy()
            for b in range(2):
                Gb = Ks[b] - out[off[b]:off[b + 1]]
                _, _, G0 = oracle.forces(Ks[b], grids[b], eps=eps)
                assert_grad_close(Gb, G0, f"engine G, trajectory {b}, eps {eps}")
    finally:
        ctx.close()


def test_field_nodes_regularised(sp):
    """The node field built with eps equals the oracle's regularised sums at
    the nodes (samples placed on the nodes, dyadic cells)."""
    grid = random_grid(8, 16, 8, seed=46)
    h = [(grid.hi - grid.lo) / n for n in grid.n]
    ax = [grid.lo + (np.arange(-1, n + 1) + 0.5) * h[a] for a, n in enumerate(grid.n)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1).astype(np.float32)
    eps = 0.03
    ctx = sp.sparkling_create(0)
    try:
        sp.sparkling_set_attraction(ctx, sp.ATTRACTION_FIELD)
        sp.sparkling_set_regularisation(ctx, eps)
        Kd = torch.from_numpy(P).cuda()
        rho = torch.from_numpy(grid.rho).cuda()
        g = sp.make_grid(rho, grid.lo, grid.hi, grid.n)
        G = torch.empty(P.shape[0], 3, dtype=torch.float64, device="cuda")
        A = torch.empty_like(G)
        sp.sparkling_grad(ctx, Kd, g, sp.ACC_KAHAN32, G=G, A=A)
        sp.sparkling_status(ctx)
        A0, phi0 = oracle.attraction_at(P.astype(np.float64), grid, eps=eps)
        err = np.abs(A.cpu().numpy() - A0)
        assert np.all(err <= 2.0 ** -23 * np.abs(A0) + 1e-13), err.max()
        _, Fa, _ = sp.sparkling_energy(ctx, Kd, g)
        assert Fa == pytest.approx(phi0.mean(), rel=1e-6)
    finally:
        ctx.close()

