"""Pins of the oracle's multi-resolution driver (Algorithm 1): the linear
interpolator between levels, the fixed-then-Barzilai-Borwein step schedule
(Sec. II-C, choice of step size), the per-level constraint scaling (Sec.
II-E) and resuming from a level.  CPU only."""
import numpy as np
import pytest

import inputs
import oracle


def grid12():
    return inputs.density_gaussian(12, 0.2, 0.05)


def spokes(nc, ns, radius, seed=0):
    return inputs.radial_spokes(nc, ns, radius, jitter=1e-3, seed=seed, dtype=np.float64)


def test_upsample_reproduces_straight_lines():
    """A shot moving at constant velocity is the same line on the fine
    raster at half the step (even samples are the coarse ones, odd ones the
    midpoints, the last one continues the last segment); each shot uses only
    its own samples; a one-sample shot is repeated."""
    rng = np.random.default_rng(1)
    Nc, d = 5, 7
    a = rng.uniform(-0.2, 0.2, size=(Nc, 1, 3)).round(3)
    v = rng.uniform(-0.01, 0.01, size=(Nc, 1, 3)).round(4)
    n = np.arange(d)[None, :, None]
    coarse = (a + n * v).reshape(-1, 3)
    fine = oracle.upsample(coarse, Nc, d).reshape(Nc, 2 * d, 3)
    m = np.arange(2 * d)[None, :, None]
    np.testing.assert_allclose(fine, a + 0.5 * m * v, rtol=0, atol=1e-15)
    one = oracle.upsample(np.array([[0.1, 0.2, 0.3], [0.4, 0.5, 0.6]]), 2, 1)
    np.testing.assert_array_equal(one, [[0.1, 0.2, 0.3]] * 2 + [[0.4, 0.5, 0.6]] * 2)


def test_fixed_steps_equal_repeated_projected_gradient_steps():
    """With every iteration on the fixed step, the driver's loop is exactly
    n_git calls of the (separately pinned) projected-gradient step."""
    g = grid12()
    Nc, Ns = 4, 32
    a, b = 1.0 / (2 * Ns), 1.0 / (8 * Ns * Ns)
    K0 = spokes(Nc, Ns, 0.95 * a * (Ns - 1) / 2)
    eta = 1.0 / (Nc * Ns)
    K, tr = oracle.optimize(K0, Nc, Ns, g, a, b, pin_index=Ns // 2, n_pit=50, n_git=4,
                            n_fixed=10, eta=eta)
    ref = K0.copy()
    for _ in range(4):
        ref = oracle.step(ref, Nc, Ns, g, eta, a, b, 0.5, Ns // 2, (0, 0, 0), 50)
    np.testing.assert_array_equal(K, ref)
    np.testing.assert_array_equal(tr, eta)


def test_barzilai_borwein_step_is_the_secant_least_squares_step():
    """After the fixed steps the step is 1/mu with mu minimising
    |mu s - y|^2 (the secant condition in the least-squares sense), s and y
    the last change of the iterate and of the gradient; found here by a
    scalar minimisation over iterates rebuilt with shorter runs."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    g = grid12()
    Nc, Ns = 4, 32
    a, b = 1.0 / (2 * Ns), 1.0 / (8 * Ns * Ns)
    K0 = spokes(Nc, Ns, 0.9 * a * (Ns - 1) / 2, seed=3)
    eta = 0.5 / (Nc * Ns)
    T = 6
    kw = dict(pin_index=-1, n_pit=60, n_fixed=T - 1, eta=eta)
    _, tr = oracle.optimize(K0, Nc, Ns, g, a, b, n_git=T, **kw)
    K1, _ = oracle.optimize(K0, Nc, Ns, g, a, b, n_git=T - 1, **kw)   # K_{T-1}
    K2, _ = oracle.optimize(K0, Nc, Ns, g, a, b, n_git=T - 2, **kw)   # K_{T-2}
    _, _, G1 = oracle.forces(K1, g)
    _, _, G2 = oracle.forces(K2, g)
    s, y = (K1 - K2).ravel(), (G1 - G2).ravel()
    res = scipy_opt.minimize_scalar(lambda mu: np.sum((mu * s - y) ** 2), bracket=(1.0, 1e4),
                                    tol=1e-14)
    assert np.all(tr[:T - 1] == eta)
    assert tr[T - 1] == pytest.approx(1.0 / res.x, rel=1e-7)
    assert tr[T - 1] != eta
    # safeguards: a BB step above eta_max is clamped
    _, tr2 = oracle.optimize(K0, Nc, Ns, g, a, b, n_git=T, eta_max=0.5 * tr[T - 1],
                             **{k: v for k, v in kw.items()})
    assert tr2[T - 1] == 0.5 * tr[T - 1]


def test_levels_scale_the_constraints_and_pin():
    """Level l (Ns / 2^l samples per shot) works under alpha 2^l and beta 4^l
    per step and pins sample pin / 2^l.  The spreading samples make both
    constraints active at every level, so the largest first and second
    differences of each level's result sit at that level's alpha and beta
    (a factor 2 off at a neighbouring level's)."""
    g = grid12()
    Nc, Ns, L = 6, 64, 2
    a, b = 1.0 / (2 * Ns), 1.0 / (8 * Ns * Ns)
    K0 = spokes(Nc, Ns >> L, 0.3)
    eta = 2.0 / (Nc * Ns)
    K, levels, tr = oracle.multires(K0, Nc, Ns, g, a, b, pin_index=Ns // 2, n_pit=400,
                                    start_level=L, n_git=25, n_fixed=20, eta=eta)
    assert tr.shape == (L + 1, 25)
    for l, Kl in zip(range(L, -1, -1), levels):
        nsl = Ns >> l
        al, bl = a * 2.0 ** l, b * 4.0 ** l
        v = oracle.violation(Kl, Nc, nsl, al, bl, 0.5, (Ns // 2) >> l, (0, 0, 0))
        assert v[0] < 0.01 * al and v[1] < 0.02 * bl, (l, v)
        assert v[3] == 0.0
        S = Kl.reshape(Nc, nsl, 3)
        d1 = np.linalg.norm(np.diff(S, axis=1), axis=2).max()
        d2 = np.linalg.norm(np.diff(S, 2, axis=1), axis=2).max()
        assert 0.95 < d1 / al < 1.01, (l, d1 / al)
        assert 0.95 < d2 / bl < 1.02, (l, d2 / bl)
    np.testing.assert_array_equal(levels[-1], K)


def test_resume_from_a_level_and_energy_decrease():
    """Stopping after a level and resuming from its up-sampled result gives
    the same final pattern as one uninterrupted run, and the run lowers the
    energy of the up-sampled initial pattern."""
    g = grid12()
    Nc, Ns, L = 4, 32, 2
    a, b = 1.0 / (2 * Ns), 1.0 / (8 * Ns * Ns)
    K0 = spokes(Nc, Ns >> L, 0.2, seed=5)
    kw = dict(pin_index=-1, n_pit=60, n_git=24, n_fixed=20, eta=1.0 / (Nc * Ns))
    K, levels, _ = oracle.multires(K0, Nc, Ns, g, a, b, start_level=L, **kw)
    up = oracle.upsample(levels[0], Nc, Ns >> L)
    K2, _, _ = oracle.multires(up, Nc, Ns, g, a, b, start_level=L - 1, **kw)
    np.testing.assert_array_equal(K, K2)
    init = oracle.upsample(oracle.upsample(K0, Nc, Ns >> L), Nc, Ns >> (L - 1))
    assert oracle.energy(K, g)[0] < oracle.energy(init, g)[0]


def test_driver_rejects_bad_arguments():
    g = grid12()
    with pytest.raises(ValueError):
        oracle.multires(np.zeros((4, 3)), 4, 12, g, 0.1, 0.1, start_level=3)   # 12 % 8 != 0
    with pytest.raises(ValueError):
        oracle.optimize(np.zeros((8, 3)), 2, 4, g, 0.1, 0.1, eta_min=0.0)
