"""Fast repulsion (SPARKLING_REPULSION_MESH): the particle-particle
particle-mesh summation through the C ABI.

* every gate is against the exact direct sums of the oracle (forces,
  energy): the mesh is an approximation, and each test states the bound its
  method error must stay within (1e-5 relative L2 of R at 24 cells, 5e-5 on
  the coarse 16-cell mesh, 2e-5 on the full-size workloads);
* the NumPy restatement of the library's mesh (tests/mesh_reference.py) is
  printed beside the result as a diagnostic only -- it follows the library's
  own design, so agreement with it proves nothing and no gate rests on it;
* a sample outside the mesh is reported, repeated calls are bitwise equal;
* an evaluation captured in a CUDA graph (after one call of the same size
  outside capture) replays bit for bit the eager result.
"""
import math

import numpy as np
import pytest

import inputs
import oracle
import mesh_reference as p3m
from gpu_util import assert_grad_close, rel_l2

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


def guard(n_cells):
    """Guard cells the library adds: the smallest g >= 4 with n_cells + 2g
    a product of 2, 3, 5 and 7."""
    g = 4
    while True:
        m = n_cells + 2 * g
        for p in (2, 3, 5, 7):
            while m % p == 0:
                m //= p
        if m == 1:
            return g
        g += 1


def mesh_ctx(sp, n_cells, sigma_cells=2.5, rc_sigmas=4.0, eps=0.0):
    c = sp.sparkling_create(0)
    sp.sparkling_set_repulsion(c, sp.REPULSION_MESH, sp.make_mesh(n_cells, sigma_cells, rc_sigmas))
    if eps:
        sp.sparkling_set_regularisation(c, eps)
    return c


def gpu_grad(sp, ctx, K, grid):
    Kd = torch.from_numpy(np.ascontiguousarray(K, np.float32)).cuda()
    rho = torch.from_numpy(grid.rho).cuda()
    g = sp.make_grid(rho, grid.lo, grid.hi, grid.n)
    G = torch.empty(K.shape[0], 3, dtype=torch.float64, device="cuda")
    R = torch.empty_like(G)
    sp.sparkling_grad(ctx, Kd, g, sp.ACC_KAHAN32, G=G, R=R)
    sp.sparkling_status(ctx)
    F = sp.sparkling_energy(ctx, Kd, g, sp.ACC_KAHAN32)
    return G.cpu().numpy(), R.cpu().numpy(), F


@pytest.mark.parametrize("eps", [0.0, 0.01])
def test_mesh_against_direct_sum(sp, eps):
    """3000 samples (a coincident pair and one sample 1.5 cells outside the
    box included), 24 mesh cells, sigma = 2.5 cells, rc = 4 sigma."""
    n_cells, sc, rs = 24, 2.5, 4.0
    rng = np.random.default_rng(61)
    K = rng.uniform(-0.5, 0.5, size=(3000, 3)).astype(np.float32)
    K[1] = K[0]
    K[7] = [0.5 + 1.5 / n_cells, 0.1, -0.2]
    K64 = K.astype(np.float64)
    N = K.shape[0]
    grid = inputs.density_gaussian(8, 0.2)
    ctx = mesh_ctx(sp, n_cells, sc, rs, eps)
    try:
        G, R, (F, Fa, Fr) = gpu_grad(sp, ctx, K, grid)
    finally:
        ctx.close()
    spec = p3m.MeshSpec(n_cells=n_cells, sigma=sc / n_cells, guard=guard(n_cells))
    S, _, eS, _ = oracle.repulsion_split(K64, spec.sigma, rc=rs * spec.sigma, eps=eps)
    Lm, eLm = p3m.mesh_long(K64, spec, eps)
    want = (S + Lm) / N
    # diagnostic only: the NumPy restatement of the same mesh design
    print(f"mesh repulsion 24 cells, eps {eps}: R rel L2 {rel_l2(R, want):.2e} against the "
          f"mesh restatement (diagnostic)")
    # the gate: method error against the exact direct sum
    A0, R0, G0 = oracle.forces(K64, grid, eps=eps)
    e = rel_l2(R, R0)
    print(f"mesh repulsion 24 cells, eps {eps}: R rel L2 {e:.2e} against the direct sum")
    assert e < 1e-5
    assert_grad_close(G, G0, "G (mesh repulsion)", rel=1e-4, atol=1e-5)
    # energy: the library's directed distance sums include the self pair of
    # every sample on both sides -- the short-range sum adds
    # g_short(eps) = eps erfc(eps/sigma) - sigma/sqrt(pi) exp(-eps^2/sigma^2),
    # the mesh potential its own approximation of g_long(eps) (as the NumPy
    # mesh does), together eps -- and the reduction removes N eps
    x = eps / spec.sigma
    g_short0 = eps * math.erfc(x) - spec.sigma / math.sqrt(math.pi) * math.exp(-x * x)
    er_p3m = eS.sum() + N * g_short0 + eLm.sum()
    Fr_p3m = (er_p3m - N * eps) / (2.0 * N * N)
    _, _, Fr0 = oracle.energy(K64, grid, eps=eps)
    print(f"mesh energy: F^r {Fr!r}, direct sum {Fr0!r}, mesh restatement {Fr_p3m!r} (diagnostic)")
    assert Fr == pytest.approx(Fr0, rel=2e-5)


def test_mesh_repeatable_and_range_error(sp):
    n_cells = 32
    rng = np.random.default_rng(62)
    K = rng.uniform(-0.45, 0.45, size=(5000, 3)).astype(np.float32)
    grid = inputs.density_gaussian(8, 0.2)
    ctx = mesh_ctx(sp, n_cells)
    try:
        G1, R1, F1 = gpu_grad(sp, ctx, K, grid)
        G2, R2, F2 = gpu_grad(sp, ctx, K, grid)
        np.testing.assert_array_equal(R1, R2)
        assert F1 == F2
        Kb = K.copy()
        Kb[3] = [0.5 + 3.5 / n_cells, 0.0, 0.0]      # beyond the guard cells
        with pytest.raises(sp.SparklingError) as e:
            gpu_grad(sp, ctx, Kb, grid)
        assert e.value.code == sp.E_RANGE
        G3, _, _ = gpu_grad(sp, ctx, K, grid)          # the context stays usable
        np.testing.assert_array_equal(G3, G1)
    finally:
        ctx.close()


def test_mesh_evaluation_captured_in_a_cuda_graph(sp):
    """The mesh path sizes and reads its short-range work list on the device,
    so a gradient call can be captured: one eager call sizes the buffers,
    then the same call captured into a CUDA graph and replayed twice (after
    K changed in place and back) gives the eager G bit for bit, and the
    replay with the changed K matches an eager call on it."""
    rng = np.random.default_rng(63)
    K = rng.uniform(-0.45, 0.45, size=(6000, 3)).astype(np.float32)
    K2 = np.clip(K + rng.normal(scale=2e-3, size=K.shape), -0.45, 0.45).astype(np.float32)
    grid = inputs.density_gaussian(8, 0.2)
    ctx = mesh_ctx(sp, 24)
    try:
        Kd = torch.from_numpy(K).cuda()
        rho = torch.from_numpy(grid.rho).cuda()
        g = sp.make_grid(rho, grid.lo, grid.hi, grid.n)
        G = torch.empty(K.shape[0], 3, dtype=torch.float64, device="cuda")
        sp.sparkling_grad(ctx, Kd, g, sp.ACC_KAHAN32, G=G)
        sp.sparkling_status(ctx)
        eager = G.cpu().numpy()
        Kd.copy_(torch.from_numpy(K2))
        sp.sparkling_grad(ctx, Kd, g, sp.ACC_KAHAN32, G=G)
        sp.sparkling_status(ctx)
        eager2 = G.cpu().numpy()
        Kd.copy_(torch.from_numpy(K))
        G.zero_()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, capture_error_mode="thread_local"):
            sp.sparkling_grad(ctx, Kd, g, sp.ACC_KAHAN32, G=G)
        graph.replay()
        torch.cuda.synchronize()
        sp.sparkling_status(ctx)
        np.testing.assert_array_equal(G.cpu().numpy(), eager)
        Kd.copy_(torch.from_numpy(K2))
        graph.replay()
        torch.cuda.synchronize()
        sp.sparkling_status(ctx)
        np.testing.assert_array_equal(G.cpu().numpy(), eager2)
        Kd.copy_(torch.from_numpy(K))
        graph.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(G.cpu().numpy(), eager)
        assert not np.array_equal(eager, eager2)
    finally:
        ctx.close()


@pytest.mark.parametrize("name,n_cells,m,sc,rs", [("diff", 128, 4096, 2.5, 4.0),
                                                   ("hr", 256, 8192, 2.5, 4.0),
                                                   ("hr", 384, 8192, 2.0, 3.5),
                                                   ("hr", 512, 8192, 2.0, 3.5)])
def test_mesh_full_size_sampled_targets(sp, name, n_cells, m, sc, rs, request):
    """Full-size workloads with the mesh repulsion (sigma sc cells, rc = rs
    sigma): R and G against the oracle's direct sums on 4096 (diff) / 8192
    (HR) random targets, R within 2e-5 relative L2 (the method-error target;
    measured 2e-7 to 3e-6)."""
    p = inputs.make_problem(name)
    ctx = mesh_ctx(sp, n_cells, sc, rs)
    try:
        Kd = torch.from_numpy(p.K).cuda()
        rho = torch.from_numpy(p.grid.rho).cuda()
        g = sp.make_grid(rho, p.grid.lo, p.grid.hi, p.grid.n)
        G = torch.empty(p.N, 3, dtype=torch.float64, device="cuda")
        R = torch.empty_like(G)
        sp.sparkling_set_timing(ctx, True)
        sp.sparkling_grad(ctx, Kd, g, sp.ACC_KAHAN32, G=G, R=R)
        sp.sparkling_status(ctx)
        t = sp.sparkling_kernel_times(ctx)
    finally:
        ctx.close()
    if name == "hr":
        _, idx, _, R0, G0 = request.getfixturevalue("hr_oracle")
    else:
        idx = np.sort(np.random.default_rng(63).choice(p.N, size=4096, replace=False))
        _, R0, G0 = oracle.forces(p.K.astype(np.float64), p.grid, targets=idx)
    eR = rel_l2(R.cpu().numpy()[idx], R0)
    eG = rel_l2(G.cpu().numpy()[idx], G0)
    print(f"mesh repulsion {name} ({n_cells} cells, sigma {sc}, rc {rs}): R rel L2 {eR:.2e}, "
          f"G rel L2 {eG:.2e}, "
          f"repulsion {t['repulsion'][0]:.1f} ms (first call, with the kernel spectra)")
    assert eR < 2e-5
    # the attraction here is the compensated-FP32 direct sum (about 1e-5 per
    # component at these grid sizes) and the mesh adds its own ~1e-6
    assert_grad_close(G.cpu().numpy()[idx], G0, f"G ({name}, mesh repulsion)", rel=2e-5,
                      atol=2e-5)


@pytest.mark.parametrize("N", [2, 33])
def test_mesh_tiny_sample_counts(sp, N):
    """The smallest problems (one pair; a ragged handful) through the mesh
    path: cell list, work items and mesh against the direct sum, within the
    coarse 16-cell mesh's method-error bound."""
    n_cells, sc, rs = 16, 2.5, 4.0
    K = np.random.default_rng(64 + N).uniform(-0.4, 0.4, size=(N, 3)).astype(np.float32)
    K64 = K.astype(np.float64)
    grid = inputs.density_gaussian(4, 0.2)
    ctx = mesh_ctx(sp, n_cells, sc, rs)
    try:
        _, R, _ = gpu_grad(sp, ctx, K, grid)
    finally:
        ctx.close()
    spec = p3m.MeshSpec(n_cells=n_cells, sigma=sc / n_cells, guard=guard(n_cells))
    S, _, _, _ = oracle.repulsion_split(K64, spec.sigma, rc=rs * spec.sigma)
    Lm, _ = p3m.mesh_long(K64, spec)
    print(f"mesh N = {N}: R rel L2 {rel_l2(R, (S + Lm) / N):.2e} against the mesh restatement "
          f"(diagnostic)")
    # the coarse 16-cell mesh's own error against the direct sum is ~1e-5
    _, R0, _ = oracle.forces(K64, grid)
    e = rel_l2(R, R0)
    print(f"mesh N = {N}: R rel L2 {e:.2e} against the direct sum")
    assert e < 5e-5
    np.testing.assert_allclose(R, R0, rtol=0, atol=5e-5)
