"""The multi-resolution driver (Algorithm 1) through the C ABI against the
oracle's driver: the linear up-sampling between levels (bit for bit), the
fixed-then-Barzilai-Borwein iterations at one resolution, every level of a
multi-resolution run (read back from the checkpoint files) and resuming from
a checkpoint."""
import os

import numpy as np
import pytest

import inputs
import oracle
from gpu_util import GRAD_ABS

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


def grid16():
    return inputs.density_gaussian(16, 0.2, 0.05)


def spokes(nc, ns, radius, seed=0):
    return inputs.radial_spokes(nc, ns, radius, jitter=1e-3, seed=seed, dtype=np.float64)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_upsample_bitwise(sp, ctx, dtype):
    rng = np.random.default_rng(51)
    for Nc, d in ((7, 33), (3, 1), (1, 2), (5, 128)):
        Kc = rng.uniform(-0.5, 0.5, size=(Nc * d, 3)).astype(dtype)
        got = sp.sparkling_upsample(ctx, torch.from_numpy(Kc).cuda(), Nc, d).cpu().numpy()
        want = oracle.upsample(Kc.astype(np.float64), Nc, d).astype(dtype)
        np.testing.assert_array_equal(got, want)


def drift_tol(steps, n_iter):
    """Each iteration moves K by eta G; a gradient within GRAD_ABS per
    component moves it by at most ~eta GRAD_ABS, and the projection does
    not expand differences: the iterates stay within the sum of those
    (factor 4 for the finitely many FISTA iterations)."""
    return 4 * GRAD_ABS * float(np.sum(steps)) + 1e-12 * n_iter


def test_optimize_fixed_then_barzilai_borwein(sp, ctx):
    """Eight shots of 64 samples, 16^3 density, FP64 samples and sums:
    20 fixed steps then Barzilai-Borwein; the steps and the iterate match."""
    g = grid16()
    Nc, Ns = 8, 64
    a, b = 1.0 / (2 * Ns), 1.0 / (8 * Ns * Ns)
    K0 = spokes(Nc, Ns, 0.9 * a * (Ns - 1) / 2, seed=3)
    eta = 0.5 / (Nc * Ns)
    n_git, n_fixed, n_pit = 26, 20, 60
    Kref, tref = oracle.optimize(K0, Nc, Ns, g, a, b, n_pit=n_pit, n_git=n_git, n_fixed=n_fixed,
                                 eta=eta)
    assert np.any(tref[n_fixed:] != eta), "the case must exercise Barzilai-Borwein steps"
    K = torch.from_numpy(K0.copy()).cuda()
    rho = torch.from_numpy(g.rho).cuda()
    grid = sp.make_grid(rho, g.lo, g.hi, g.n)
    proj = sp.make_proj(a, b, 0.5, n_pit)
    sched = sp.make_schedule(eta, n_git, n_fixed)
    steps = sp.sparkling_optimize(ctx, K, Nc, Ns, grid, proj, sched, sp.ACC_FP64)
    np.testing.assert_array_equal(steps[:n_fixed], eta)
    np.testing.assert_allclose(steps, tref, rtol=1e-3)
    np.testing.assert_allclose(K.cpu().numpy(), Kref, rtol=0, atol=drift_tol(tref, n_git))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_multires_levels_checkpoints_and_resume(sp, ctx, tmp_path, dtype):
    """Three levels (16, 32, 64 samples per shot) with a pinned TE sample:
    every level's checkpoint matches the oracle's result of that level; a
    run resumed from the up-sampled level-2 checkpoint reproduces the
    uninterrupted run bit for bit."""
    g = grid16()
    Nc, Ns, L = 6, 64, 2
    a, b = 1.0 / (2 * Ns), 1.0 / (8 * Ns * Ns)
    K0 = spokes(Nc, Ns >> L, 0.25, seed=7)
    eta = 1.0 / (Nc * Ns)
    kw = dict(n_pit=80, n_git=22, n_fixed=20, eta=eta)
    Kref, levels, tref = oracle.multires(K0.astype(dtype).astype(np.float64), Nc, Ns, g, a, b,
                                         pin_index=Ns // 2, start_level=L, **kw)
    rho = torch.from_numpy(g.rho).cuda()
    grid = sp.make_grid(rho, g.lo, g.hi, g.n)
    proj = sp.make_proj(a, b, 0.5, kw["n_pit"], Ns // 2)
    sched = sp.make_schedule(eta, kw["n_git"], kw["n_fixed"])
    K = torch.zeros(Nc * Ns, 3, dtype=torch.from_numpy(K0.astype(dtype)).dtype, device="cuda")
    K[:Nc * (Ns >> L)] = torch.from_numpy(K0.astype(dtype)).cuda()
    prefix = str(tmp_path / "run")
    steps = sp.sparkling_multires(ctx, K, Nc, Ns, grid, proj, sched, L, sp.ACC_FP64, prefix)
    out = K.cpu().numpy().astype(np.float64)
    f32 = dtype == np.float32
    for l, Kl in zip(range(L, -1, -1), levels):
        level, nc, nsl, arr = sp.read_checkpoint(f"{prefix}_level{l}.bin")
        assert (level, nc, nsl) == (l, Nc, Ns >> l)
        tol = drift_tol(tref[:L - l + 1], kw["n_git"] * (L - l + 1))
        if f32:
            tol += 2e-6 * (L - l + 1)      # float rounding of every iterate
        np.testing.assert_allclose(arr.astype(np.float64), Kl, rtol=0, atol=tol)
        np.testing.assert_array_equal(arr[(Ns // 2 >> l)::nsl], 0.0)   # pinned sample
    np.testing.assert_allclose(steps, tref, rtol=1e-3)
    np.testing.assert_array_equal(out, sp.read_checkpoint(f"{prefix}_level0.bin")[3])

    # resume from the level-2 checkpoint
    _, _, _, k2 = sp.read_checkpoint(f"{prefix}_level2.bin")
    up = sp.sparkling_upsample(ctx, torch.from_numpy(k2).cuda(), Nc, Ns >> L)
    K2 = torch.zeros_like(K)
    K2[:up.shape[0]] = up
    sp.sparkling_multires(ctx, K2, Nc, Ns, grid, proj, sched, L - 1, sp.ACC_FP64)
    np.testing.assert_array_equal(K2.cpu().numpy(), K.cpu().numpy())


def test_checkpoint_io_error_reported(sp, ctx, tmp_path):
    g = grid16()
    Nc, Ns = 2, 16
    rho = torch.from_numpy(g.rho).cuda()
    grid = sp.make_grid(rho, g.lo, g.hi, g.n)
    K = torch.from_numpy(spokes(Nc, Ns, 0.1)).cuda()
    sched = sp.make_schedule(1e-3, 1, 20)
    with pytest.raises(sp.SparklingError) as e:
        sp.sparkling_multires(ctx, K, Nc, Ns, grid, sp.make_proj(0.05, 0.01), sched, 0,
                              checkpoint_prefix=os.path.join(str(tmp_path), "missing", "x"))
    assert e.value.code == sp.E_IO
