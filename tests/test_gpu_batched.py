"""The batched persistent step (B trajectories of uneven size: one engine
launch whose work list also holds the symmetric repulsion items -- the
default -- or the symmetric repulsion kernel followed by the engine;
optionally replayed from a CUDA graph) against the oracle."""
import numpy as np
import pytest

import inputs
import oracle
from gpu_util import GRAD_ABS, PROJ_F32_ROUND, assert_grad_close, proj_tol_f32

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


@pytest.fixture(scope="module")
def ctx(sp):
    c = sp.sparkling_create(0)
    yield c
    c.close()


def make_batch(seed, shots, Ns, grid_shapes, dtype):
    rng = np.random.default_rng(seed)
    Ks, grids, projs, etas = [], [], [], []
    for b, (nc, shape) in enumerate(zip(shots, grid_shapes)):
        K = np.cumsum(rng.normal(scale=3e-3, size=(nc, Ns, 3)), axis=1).reshape(-1, 3)
        K = np.clip(K + rng.uniform(-0.2, 0.2, size=(1, 3)), -0.45, 0.45)
        Ks.append(K.astype(dtype))
        nx, ny, nz = shape
        rho = rng.uniform(0.0, 1.0, size=(nz, ny, nx))
        grids.append(inputs.Grid(shape, -0.5, 0.5, (rho / rho.sum()).astype(np.float32)))
        a = (0.5 + rng.uniform()) / (2 * Ns)
        pb = (0.5 + rng.uniform()) / (8 * Ns * Ns)
        projs.append(inputs.Proj(a, pb, 0.5, pin_index=(Ns // 2 if b % 2 else -1), n_iter=40))
        etas.append(1.0 / (nc * Ns))
    return Ks, grids, projs, etas


def run_batched(sp, ctx, Ks, grids, projs, etas, Ns, graph, calls=1, one_launch=True):
    off = np.concatenate([[0], np.cumsum([k.shape[0] for k in Ks])])
    K = torch.from_numpy(np.concatenate(Ks)).cuda()
    rhos = [torch.from_numpy(g.rho).cuda() for g in grids]
    gs = [sp.make_grid(r, g.lo, g.hi, g.n) for r, g in zip(rhos, grids)]
    ps = [sp.make_proj(p.alpha, p.beta, p.box, p.n_iter, p.pin_index, p.pin) for p in projs]
    outs = []
    for _ in range(calls):
        sp.sparkling_step_batched(ctx, K, off, Ns, gs, etas, ps, graph=graph, one_launch=one_launch)
        sp.sparkling_status(ctx)
        outs.append(K.cpu().numpy().copy())
    return off, outs


def oracle_step(K, g, p, eta, Ns):
    return oracle.step(K, K.shape[0] // Ns, Ns, g, eta, p.alpha, p.beta, p.box, p.pin_index, p.pin,
                       p.n_iter)


@pytest.mark.parametrize("one_launch", [False, True])
@pytest.mark.parametrize("dtype,mixed", [(np.float64, False), (np.float32, False),
                                         (np.float32, True)])
def test_batched_step_matches_oracle_every_sample(sp, dtype, mixed, one_launch):
    """Five trajectories (1..21 shots of 64 samples, ragged tiles), grids of
    different shapes (rows not a multiple of 4, a one-cell grid), per-
    trajectory alpha, beta, eta and pins; one eager call.  FP32 samples with
    the default FP64 projection and with the opt-in mixed form."""
    Ns = 64
    shots = [3, 1, 21, 7, 2]
    shapes = [(9, 5, 4), (1, 1, 1), (16, 16, 16), (13, 3, 7), (4, 4, 4)]
    Ks, grids, projs, etas = make_batch(1, shots, Ns, shapes, dtype)
    c = sp.sparkling_create(0)
    try:
        if mixed:
            sp.sparkling_set_projection(c, sp.PROJECTION_MIXED)
        off, outs = run_batched(sp, c, Ks, grids, projs, etas, Ns, graph=False,
                                one_launch=one_launch)
    finally:
        c.close()
    out = outs[0]
    for b in range(len(Ks)):
        ref = oracle_step(Ks[b], grids[b], projs[b], etas[b], Ns)
        got = out[off[b]:off[b + 1]].astype(np.float64)
        # the step moves by eta * G: a gradient within GRAD_ABS per component
        # moves the result by at most ~eta * GRAD_ABS (factor 4 for the
        # finitely many FISTA iterations), plus the FP32 output rounding (one
        # ulp of 1/2) or the mixed form's bound
        tol = 4 * etas[b] * GRAD_ABS
        if dtype == np.float32:
            tol += proj_tol_f32(ref, Ks[b]) if mixed else PROJ_F32_ROUND
        want = ref if dtype == np.float64 else ref.astype(np.float32).astype(np.float64)
        np.testing.assert_allclose(got, want, rtol=0, atol=tol)


@pytest.mark.parametrize("one_launch", [False, True])
def test_batched_gradient_recovered_from_unconstrained_step(sp, ctx, one_launch):
    """With alpha = beta = inf and a loose box the projection is the identity,
    so K' = K - eta G exposes the engine's gradient: G = (K - K') / eta."""
    Ns = 128
    shots = [9, 2, 17]
    shapes = [(20, 10, 8), (7, 7, 7), (32, 8, 4)]
    Ks, grids, projs, _ = make_batch(2, shots, Ns, shapes, np.float64)
    projs = [inputs.Proj(INF, INF, 10.0, n_iter=3) for _ in projs]
    etas = [1.0, 0.5, 2.0]
    off, outs = run_batched(sp, ctx, Ks, grids, projs, etas, Ns, graph=False,
                            one_launch=one_launch)
    for b in range(3):
        G = (Ks[b] - outs[0][off[b]:off[b + 1]]) / etas[b]
        _, _, G0 = oracle.forces(Ks[b], grids[b])
        assert_grad_close(G, G0, f"engine G of trajectory {b}")


@pytest.mark.parametrize("one_launch", [False, True])
def test_batched_graph_replay_is_bitwise_the_eager_step(sp, ctx, one_launch):
    """Call 1 runs eagerly, call 2 captures the device work into a CUDA graph,
    call 3 replays it; each matches an eager chain bit for bit."""
    Ns = 64
    Ks, grids, projs, etas = make_batch(3, [4, 6, 3], Ns, [(8, 8, 8), (6, 5, 4), (10, 3, 3)],
                                        np.float32)
    _, eager = run_batched(sp, ctx, Ks, grids, projs, etas, Ns, graph=False, calls=3,
                           one_launch=one_launch)
    ctx2 = sp.sparkling_create(0)
    try:
        _, graphed = run_batched(sp, ctx2, Ks, grids, projs, etas, Ns, graph=True, calls=3,
                                 one_launch=one_launch)
    finally:
        ctx2.close()
    for a, b in zip(eager, graphed):
        np.testing.assert_array_equal(a, b)


def test_batched_workload_sampled(sp, ctx):
    """The batched workload at full size: 64 trajectories of 512-sample shots,
    N_b = 512 * U{32..512}, 64^3 Gaussian densities, uneven alpha/beta; per
    trajectory 2 shots of the step's projection checked against the oracle
    projection of K - eta G, with G from sparkling_grad on that trajectory
    (the engine's own gradient is checked against the oracle in
    test_batched_workload_gradient)."""
    probs = inputs.make_batched(seed=0)
    Ns = 512
    off = np.concatenate([[0], np.cumsum([p.N for p in probs])])
    K = torch.from_numpy(np.concatenate([p.K for p in probs])).cuda()
    K0 = K.clone()
    rhos = [torch.from_numpy(p.grid.rho).cuda() for p in probs]
    gs = [sp.make_grid(r, p.grid.lo, p.grid.hi, p.grid.n) for r, p in zip(rhos, probs)]
    ps = [sp.make_proj(p.proj.alpha, p.proj.beta, p.proj.box, p.proj.n_iter) for p in probs]
    sp.sparkling_step_batched(ctx, K, off, Ns, gs, [p.eta for p in probs], ps, graph=False)
    sp.sparkling_status(ctx)
    rng = np.random.default_rng(7)
    for b in rng.choice(len(probs), size=6, replace=False):
        p = probs[b]
        Kb = K0[off[b]:off[b + 1]].contiguous()
        G = sp.sparkling_grad(ctx, Kb, gs[b], G=torch.empty(p.N, 3, dtype=torch.float64,
                                                             device="cuda"))
        sp.sparkling_status(ctx)
        Kh = Kb.cpu().numpy().astype(np.float64)
        half = Kh - p.eta * G.cpu().numpy()
        out = K[off[b]:off[b + 1]].cpu().numpy().astype(np.float64)
        for c in rng.choice(p.Nc, size=2, replace=False):
            sl = slice(c * Ns, (c + 1) * Ns)
            ref = oracle.project(half[sl], 1, Ns, p.proj.alpha, p.proj.beta, p.proj.box, -1,
                                 (0.0, 0.0, 0.0), p.proj.n_iter)
            np.testing.assert_allclose(out[sl], ref.astype(np.float32), rtol=0,
                                       atol=PROJ_F32_ROUND + 4 * p.eta * GRAD_ABS)


@pytest.mark.parametrize("one_launch", [False, True])
def test_batched_workload_gradient(sp, ctx, one_launch):
    """The engine's gradient on the full batched workload (64 trajectories,
    9.07M samples) against the oracle on 64 random targets of every
    trajectory, with the repulsion in its own kernel or as items of the one
    engine launch.  alpha = beta = inf and a loose box make the projection the
    identity, so K' = K - eta G exposes G = (K - K') / eta; K in FP64 keeps
    that difference exact to ~1e-16 / eta."""
    probs = inputs.make_batched(seed=0)
    Ns = 512
    off = np.concatenate([[0], np.cumsum([p.N for p in probs])])
    K64 = np.concatenate([p.K for p in probs]).astype(np.float64)
    K = torch.from_numpy(K64).cuda()
    rhos = [torch.from_numpy(p.grid.rho).cuda() for p in probs]
    gs = [sp.make_grid(r, p.grid.lo, p.grid.hi, p.grid.n) for r, p in zip(rhos, probs)]
    ps = [sp.make_proj(INF, INF, 10.0, 2) for _ in probs]
    etas = [p.eta for p in probs]
    sp.sparkling_step_batched(ctx, K, off, Ns, gs, etas, ps, graph=False, one_launch=one_launch)
    sp.sparkling_status(ctx)
    out = K.cpu().numpy()
    rng = np.random.default_rng(8)
    for b, p in enumerate(probs):
        idx = np.sort(rng.choice(p.N, size=64, replace=False))
        Kb = K64[off[b]:off[b + 1]]
        G = (Kb[idx] - out[off[b]:off[b + 1]][idx]) / etas[b]
        _, _, G0 = oracle.forces(Kb, p.grid, targets=idx)
        assert_grad_close(G, G0, f"engine G of trajectory {b} (N = {p.N}), 64 targets")
