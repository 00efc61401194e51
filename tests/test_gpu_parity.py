"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Small cases are compared element by element over every sample; they span
several target tiles (1024 targets each), several pipeline stages, ragged
tails and grid rows whose length is not a multiple of 4.  Full-size
workloads are compared on sampled targets / shots that the oracle computes
one by one.
"""
import numpy as np
import pytest

import inputs
import oracle
from gpu_util import PROJ_F32_ROUND, assert_grad_close, proj_tol_f32, rel_l2

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


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def gpu_grad(sp, ctx, K, grid, acc=0, out_dtype=torch.float64):
    Kd = dev(K)
    rho = dev(grid.rho)
    g = sp.make_grid(rho, grid.lo, grid.hi, grid.n)
    G = torch.empty(K.shape, dtype=out_dtype, device="cuda")
    A = torch.empty_like(G)
    R = torch.empty_like(G)
    sp.sparkling_grad(ctx, Kd, g, acc, G=G, A=A, R=R)
    sp.sparkling_status(ctx)
    return G.cpu().numpy(), A.cpu().numpy(), R.cpu().numpy()


def random_grid(nx, ny, nz, seed, lo=-0.5, hi=0.5):
    rho = np.random.default_rng(seed).uniform(0.0, 1.0, size=(nz, ny, nx))
    rho = (rho / rho.sum()).astype(np.float32)
    return inputs.Grid((nx, ny, nz), lo, hi, rho)


@pytest.mark.parametrize("acc", [0, 1])
def test_grad_tiny_every_sample(sp, ctx, acc):
    p = inputs.make_problem("tiny")
    A0, R0, G0 = oracle.forces(p.K, p.grid)
    G, A, R = gpu_grad(sp, ctx, p.K, p.grid, acc)
    assert_grad_close(A, A0, "A")
    assert_grad_close(R, R0, "R")
    assert_grad_close(G, G0, "G")


@pytest.mark.parametrize("N,shape,lo,hi,dt", [
    (3000, (13, 7, 5), -0.5, 0.5, np.float64),      # 3 tiles, ragged tile and rows
    (2049, (5, 9, 4), -0.3, 0.6, np.float32),       # one target past two tiles
    (1029, (1, 3, 2), -0.5, 0.5, np.float32),         # nx = 1
    (5000, (1000, 3, 2), -0.5, 0.5, np.float32),    # rows of 1000 points, 4 rows per stage
    (2, (6, 5, 4), -0.5, 0.5, np.float64),          # the smallest N
])
def test_grad_ragged_shapes(sp, ctx, N, shape, lo, hi, dt):
    rng = np.random.default_rng(N)
    K = rng.uniform(lo, hi, size=(N, 3)).astype(dt)
    grid = random_grid(*shape, seed=N + 1, lo=lo, hi=hi)
    A0, R0, G0 = oracle.forces(K, grid)
    for out in (torch.float64, torch.float32):
        G, A, R = gpu_grad(sp, ctx, K, grid, 0, out)
        assert_grad_close(A, A0, "A")
        assert_grad_close(R, R0, "R")
        assert_grad_close(G, G0, "G")


def test_grad_longest_grid_rows(sp, ctx):
    """Grid rows of the largest supported length (nx = 4096: one row fills a
    pipeline stage) and a ragged target tail."""
    rng = np.random.default_rng(71)
    K = rng.uniform(-0.5, 0.5, size=(1500, 3)).astype(np.float32)
    grid = random_grid(4096, 3, 2, seed=72)
    A0, R0, G0 = oracle.forces(K, grid)
    G, A, R = gpu_grad(sp, ctx, K, grid)
    assert_grad_close(A, A0, "A")
    assert_grad_close(R, R0, "R")
    # uniform samples against a uniform-ish density: A and R nearly cancel,
    # and G's relative error is A's and R's scaled by the subtraction's
    # condition number (|A| + |R|) / (2 |G|)
    cond = (np.linalg.norm(A0) + np.linalg.norm(R0)) / np.linalg.norm(G0) / 2
    assert_grad_close(G, G0, f"G (condition {cond:.0f})", rel=1e-5 * max(cond, 1.0))


def test_grad_many_source_blocks_and_tiles(sp, ctx):
    """N = 9000: 9 tiles, 9 repulsion source blocks (the last ragged), spokes."""
    K = inputs.radial_spokes(18, 500, 0.23, jitter=1e-3, seed=3, dtype=np.float32)
    grid = inputs.density_gaussian(40, 0.15, 0.05)
    A0, R0, G0 = oracle.forces(K, grid)
    G, A, R = gpu_grad(sp, ctx, K, grid)
    assert_grad_close(G, G0, "G")
    assert_grad_close(R, R0, "R")


def test_grad_degenerate_cases(sp, ctx):
    """Coincident samples, a sample on a grid point and a one-cell grid:
    zero-distance terms contribute nothing (same reading as the oracle)."""
    grid = inputs.Grid((1, 1, 1), -0.5, 0.5, np.ones((1, 1, 1), np.float32))
    K = np.array([[0.1, 0.2, 0.3], [0.1, 0.2, 0.3], [-0.2, 0.0, 0.1], [0.0, 0.0, 0.0]])
    A0, R0, G0 = oracle.forces(K, grid)
    G, A, R = gpu_grad(sp, ctx, K, grid)
    assert_grad_close(G, G0, "G", atol=1e-6)
    np.testing.assert_array_equal(A[3], [0.0, 0.0, 0.0])   # on the grid point
    # N = 2 closed form: R_1 = u/2.
    K2 = np.array([[0.25, -0.1, 0.0], [-0.05, 0.3, 0.2]])
    _, _, R2 = gpu_grad(sp, ctx, K2, grid)
    u = (K2[0] - K2[1]) / np.linalg.norm(K2[0] - K2[1])
    np.testing.assert_allclose(R2[0], 0.5 * u, atol=1e-7)
    np.testing.assert_allclose(R2[1], -0.5 * u, atol=1e-7)


def test_grad_repeatable_bitwise(sp, ctx):
    p = inputs.make_problem("tiny")
    G1, _, _ = gpu_grad(sp, ctx, p.K, p.grid)
    G2, _, _ = gpu_grad(sp, ctx, p.K, p.grid)
    np.testing.assert_array_equal(G1, G2)


@pytest.mark.parametrize("acc", [0, 1])
def test_energy_tiny(sp, ctx, acc):
    p = inputs.make_problem("tiny")
    F0, Fa0, Fr0 = oracle.energy(p.K, p.grid)
    Kd = dev(p.K)
    g = sp.make_grid(dev(p.grid.rho), p.grid.lo, p.grid.hi, p.grid.n)
    F, Fa, Fr = sp.sparkling_energy(ctx, Kd, g, acc)
    assert Fa == pytest.approx(Fa0, rel=1e-6)
    assert Fr == pytest.approx(Fr0, rel=1e-6)
    assert F == pytest.approx(F0, abs=1e-6 * (Fa0 + Fr0))
    assert sp.sparkling_energy(ctx, Kd, g, acc) == (F, Fa, Fr)   # fixed reduction order


def test_energy_ragged(sp, ctx):
    rng = np.random.default_rng(21)
    K = rng.uniform(-0.5, 0.5, size=(2500, 3)).astype(np.float32)
    grid = random_grid(11, 6, 9, seed=22)
    F0, Fa0, Fr0 = oracle.energy(K, grid)
    g = sp.make_grid(dev(grid.rho), grid.lo, grid.hi, grid.n)
    F, Fa, Fr = sp.sparkling_energy(ctx, dev(K), g)
    assert Fa == pytest.approx(Fa0, rel=1e-6)
    assert Fr == pytest.approx(Fr0, rel=1e-6)


def proj_of(pp: inputs.Proj, sp, **kw):
    d = dict(alpha=pp.alpha, beta=pp.beta, box=pp.box, n_iter=pp.n_iter, pin_index=pp.pin_index,
             pin=pp.pin)
    d.update(kw)
    return sp.make_proj(**d)


def oracle_project(K, Nc, Ns, pr):
    return oracle.project(K, Nc, Ns, pr.alpha, pr.beta, pr.box, pr.pin_index, tuple(pr.pin),
                          pr.n_iter, pr.tol, pr.margin, max(pr.check_every, 1))


def test_project_tiny_fixed_iterations(sp, ctx):
    p = inputs.make_problem("tiny")
    pr = proj_of(p.proj, sp)
    ref = oracle_project(p.K, p.Nc, p.Ns, pr)
    Kd = dev(p.K)
    sp.sparkling_project(ctx, Kd, p.Nc, p.Ns, pr)
    sp.sparkling_status(ctx)
    np.testing.assert_allclose(Kd.cpu().numpy(), ref, rtol=0, atol=1e-11)


@pytest.mark.parametrize("Nc,Ns,dt,kw", [
    (7, 33, np.float64, dict(pin_index=16, pin=(0.0, 0.01, -0.02))),   # ragged Ns, pin
    (5, 1, np.float64, dict()),                                         # no differences
    (5, 2, np.float64, dict(beta=float("inf"))),                        # amplitude only
    (4, 3, np.float64, dict(alpha=float("inf"))),                       # slew only
    (9, 512, np.float32, dict(pin_index=256)),                          # f32, one sample/thread
    (3, 1500, np.float64, dict()),                                      # > 1024 samples per shot
    (3, 2560, np.float32, dict(pin_index=1280)),                        # state in global memory
    (2, 65536, np.float64, dict(pin_index=32768)),                      # the largest Ns
    (2, 65536, np.float32, dict()),
])
def test_project_shapes(sp, ctx, Nc, Ns, dt, kw):
    rng = np.random.default_rng(Nc * 1000 + Ns)
    K = np.cumsum(rng.normal(scale=2e-3, size=(Nc, Ns, 3)), axis=1).reshape(-1, 3)
    K = np.clip(K, -0.45, 0.45).astype(dt)
    base = dict(alpha=1.0 / (2 * Ns), beta=1.0 / (8 * Ns * Ns), n_iter=60)
    base.update(kw)
    pr = sp.make_proj(**base)
    ref = oracle_project(K, Nc, Ns, pr)
    Kd = dev(K)
    v = sp.sparkling_project(ctx, Kd, Nc, Ns, pr, want_violation=True)
    out = Kd.cpu().numpy().astype(np.float64)
    if dt == np.float64:
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-11)
    else:       # FP64 iteration (the default), one rounding to FP32
        np.testing.assert_allclose(out, ref.astype(np.float32), rtol=0, atol=PROJ_F32_ROUND)
    vref = oracle.violation(out, Nc, Ns, pr.alpha, pr.beta, pr.box, pr.pin_index, tuple(pr.pin))
    np.testing.assert_allclose(v, vref, rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("Nc,Ns,kw", [
    (9, 512, dict(pin_index=256)),
    (3, 2560, dict(pin_index=1280)),
    (2, 65536, dict()),
])
def test_project_mixed_precision_opt_in(sp, Nc, Ns, kw):
    """PROJECTION_MIXED: FP32 samples iterate in FP32 on the displacement;
    gated by the mixed form's bound.  FP64 samples keep the FP64 iteration
    in that mode too."""
    rng = np.random.default_rng(Nc * 1000 + Ns)
    K = np.cumsum(rng.normal(scale=2e-3, size=(Nc, Ns, 3)), axis=1).reshape(-1, 3)
    K = np.clip(K, -0.45, 0.45).astype(np.float32)
    base = dict(alpha=1.0 / (2 * Ns), beta=1.0 / (8 * Ns * Ns), n_iter=60)
    base.update(kw)
    pr = sp.make_proj(**base)
    ref = oracle_project(K, Nc, Ns, pr)
    c = sp.sparkling_create(0)
    try:
        sp.sparkling_set_projection(c, sp.PROJECTION_MIXED)
        Kd = dev(K)
        sp.sparkling_project(c, Kd, Nc, Ns, pr)
        sp.sparkling_status(c)
        np.testing.assert_allclose(Kd.cpu().numpy(), ref.astype(np.float32), rtol=0,
                                   atol=proj_tol_f32(ref, K))
        K64 = dev(K.astype(np.float64))
        sp.sparkling_project(c, K64, Nc, Ns, pr)
        sp.sparkling_status(c)
        np.testing.assert_allclose(K64.cpu().numpy(), ref, rtol=0, atol=1e-11)
    finally:
        c.close()


def test_project_converged_feasible(sp, ctx):
    """Converged mode: the FP64 result is feasible to 1e-9 (margin 1e-4
    shrinks the target set) and close to the oracle's converged result."""
    rng = np.random.default_rng(5)
    Nc, Ns = 6, 40
    K = np.cumsum(rng.normal(scale=5e-3, size=(Nc, Ns, 3)), axis=1).reshape(-1, 3)
    pr = sp.make_proj(alpha=0.004, beta=0.0008, n_iter=200000, tol=1e-10, margin=1e-4,
                      check_every=20)
    Kd = dev(K)
    v = sp.sparkling_project(ctx, Kd, Nc, Ns, pr, want_violation=True)
    assert max(v) <= 1e-9
    ref = oracle_project(K, Nc, Ns, pr)
    np.testing.assert_allclose(Kd.cpu().numpy(), ref, atol=1e-7)


def test_project_idempotent_on_feasible(sp, ctx):
    t = np.linspace(0, 1, 64)[:, None]
    K = 0.2 * np.hstack([np.sin(3 * t), np.cos(2 * t), t - 0.5])
    d1 = np.linalg.norm(np.diff(K, axis=0), axis=1).max()
    d2 = np.linalg.norm(np.diff(K, 2, axis=0), axis=1).max()
    pr = sp.make_proj(alpha=1.01 * d1, beta=1.01 * d2, n_iter=50)
    Kd = dev(K)
    sp.sparkling_project(ctx, Kd, 1, 64, pr)
    np.testing.assert_array_equal(Kd.cpu().numpy(), K)


@pytest.mark.parametrize("path", ["kernels", "engine"])
def test_step_tiny(sp, path):
    """The projected-gradient step through either device path of
    sparkling_step: the kernels in turn, or the one-launch persistent engine
    (which the library takes for large steps)."""
    p = inputs.make_problem("tiny")
    pr = proj_of(p.proj, sp)
    ref = oracle.step(p.K, p.Nc, p.Ns, p.grid, p.eta, pr.alpha, pr.beta, pr.box, pr.pin_index,
                      tuple(pr.pin), pr.n_iter)
    c = sp.sparkling_create(0)
    try:
        sp.sparkling_set_step_path(c, path)
        sp.sparkling_set_timing(c, True)
        Kd = dev(p.K)
        g = sp.make_grid(dev(p.grid.rho), p.grid.lo, p.grid.hi, p.grid.n)
        sp.sparkling_step(c, Kd, p.Nc, p.Ns, g, p.eta, pr)
        sp.sparkling_status(c)
        t = sp.sparkling_kernel_times(c)
    finally:
        c.close()
    assert (t["engine"][1] > 0) == (path == "engine") and t["step"][1] == 1
    np.testing.assert_allclose(Kd.cpu().numpy(), ref, rtol=0, atol=1e-8)


def test_engine_step_after_a_gradient_call(sp):
    """The engine keeps its planned work list in the context's workspace
    across steps; a gradient call in between carves the same workspace, so
    the next step must plan and upload its list again: the two steps agree
    bit for bit and with the oracle."""
    p = inputs.make_problem("tiny")
    pr = proj_of(p.proj, sp)
    ref = oracle.step(p.K, p.Nc, p.Ns, p.grid, p.eta, pr.alpha, pr.beta, pr.box, pr.pin_index,
                      tuple(pr.pin), pr.n_iter)
    c = sp.sparkling_create(0)
    try:
        sp.sparkling_set_step_path(c, "engine")
        g = sp.make_grid(dev(p.grid.rho), p.grid.lo, p.grid.hi, p.grid.n)
        outs = []
        for _ in range(2):
            Kd = dev(p.K)
            sp.sparkling_step(c, Kd, p.Nc, p.Ns, g, p.eta, pr)
            sp.sparkling_status(c)
            outs.append(Kd.cpu().numpy())
            # a larger gradient call overwrites the start of the workspace
            Kb = dev(np.random.default_rng(5).uniform(-0.4, 0.4, size=(20000, 3)))
            sp.sparkling_grad(c, Kb, g)
            sp.sparkling_status(c)
    finally:
        c.close()
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_allclose(outs[1], ref, rtol=0, atol=1e-8)


def test_invalid_pointers_rejected(sp, ctx):
    """Host memory passed as a device pointer is refused before any launch."""
    K = torch.zeros(16, 3, dtype=torch.float64)
    g = sp.make_grid(torch.ones(2, 2, 2, device="cuda"), -0.5, 0.5)
    import ctypes
    G = torch.empty(16, 3, dtype=torch.float64, device="cuda")
    code = sp.lib().sparkling_grad(ctx.handle, ctypes.c_void_p(K.data_ptr()), 1, 16,
                                   ctypes.byref(g), 0, ctypes.c_void_p(G.data_ptr()), 1, None, None,
                                   None)
    assert code == sp.E_INVAL


def test_nonfinite_input_reported(sp, ctx):
    p = inputs.make_problem("tiny")
    K = p.K.copy()
    K[17, 1] = np.nan
    g = sp.make_grid(dev(p.grid.rho), p.grid.lo, p.grid.hi, p.grid.n)
    with pytest.raises(sp.SparklingError) as e:
        sp.sparkling_energy(ctx, dev(K), g)
    assert e.value.code == sp.E_NONFINITE
    sp.sparkling_energy(ctx, dev(p.K), g)          # the context stays usable
    rho = p.grid.rho.copy()
    rho[0, 0, 0] = -1.0
    g2 = sp.make_grid(dev(rho), p.grid.lo, p.grid.hi, p.grid.n)
    sp.sparkling_grad(ctx, dev(p.K), g2)
    with pytest.raises(sp.SparklingError) as e:
        sp.sparkling_status(ctx)
    assert e.value.code == sp.E_NONFINITE


def test_plain_fp64_accumulation_mode(sp, ctx):
    """ACC_FP64_PAIR, the plain FP64-accumulate form (every attraction pair
    term added in FP64): A, R, G and the energy against the oracle on a
    ragged problem (3 target tiles, rows not a multiple of 4), in every
    attraction shape."""
    rng = np.random.default_rng(41)
    K = rng.uniform(-0.5, 0.5, size=(2500, 3)).astype(np.float32)
    grid = random_grid(11, 6, 9, seed=42)
    A0, R0, G0 = oracle.forces(K.astype(np.float64), grid)
    _, Fa0, Fr0 = oracle.energy(K.astype(np.float64), grid)
    for v in range(3):
        c = sp.sparkling_create(0)
        try:
            sp.sparkling_set_shape(c, "attraction", v)
            G, A, R = gpu_grad(sp, c, K, grid, acc=sp.ACC_FP64_PAIR)
            g = sp.make_grid(dev(grid.rho), grid.lo, grid.hi, grid.n)
            F, Fa, Fr = sp.sparkling_energy(c, dev(K), g, sp.ACC_FP64_PAIR)
        finally:
            c.close()
        assert_grad_close(A, A0, f"A (plain FP64 accumulation, shape {v})")
        assert_grad_close(R, R0, f"R (plain FP64 accumulation, shape {v})")
        assert_grad_close(G, G0, f"G (plain FP64 accumulation, shape {v})")
        assert Fa == pytest.approx(Fa0, rel=1e-6)
        assert Fr == pytest.approx(Fr0, rel=1e-6)


def test_step_timing_scope(sp):
    """With timing on, every sparkling_step is also timed as one STEP scope
    that holds its launches (pack, attraction, repulsion, combine,
    projection)."""
    p = inputs.make_problem("tiny")
    pr = proj_of(p.proj, sp)
    c = sp.sparkling_create(0)
    try:
        g = sp.make_grid(dev(p.grid.rho), p.grid.lo, p.grid.hi, p.grid.n)
        Kd = dev(p.K)
        sp.sparkling_step(c, Kd, p.Nc, p.Ns, g, p.eta, pr)          # tuning outside the timing
        sp.sparkling_status(c)
        sp.sparkling_set_timing(c, True)
        sp.sparkling_kernel_times(c, reset=True)
        for _ in range(3):
            sp.sparkling_step(c, Kd, p.Nc, p.Ns, g, p.eta, pr)
        sp.sparkling_status(c)
        t = sp.sparkling_kernel_times(c, reset=True)
    finally:
        c.close()
    ms, n = t["step"]
    assert n == 3 and ms > 0
    inner = sum(t[k][0] for k in ("pack", "attraction", "repulsion", "combine", "project"))
    assert all(t[k][1] == 3 for k in ("attraction", "repulsion", "project"))
    assert ms >= 0.9 * inner, (ms, inner)
