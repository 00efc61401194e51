"""Pins of the FP64 oracle's forces and energy against closed forms,
invariants, finite differences and a high-precision derivative.

Every test here runs on the CPU.  Each targets a plausible mistake:
a wrong sign, a dropped 1/N, an off-by-half grid coordinate, transposed
density axes, a missing density weight, a wrong energy normalisation.
"""
import json
import math
import os

import numpy as np
import pytest

import inputs
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def one_cell(lo=-0.5, hi=0.5):
    return inputs.Grid((1, 1, 1), lo, hi, np.ones((1, 1, 1), np.float32))


def random_grid(shape_xyz, seed, lo=-0.5, hi=0.5):
    nx, ny, nz = shape_xyz
    rho = np.random.default_rng(seed).uniform(0.1, 1.0, size=(nz, ny, nx))
    rho = (rho / rho.sum()).astype(np.float32)
    return inputs.Grid((nx, ny, nz), lo, hi, rho)


def test_cube_corners_golden():
    """Closed form for 8 samples on cube corners (tests/golden/cube_corners.json)."""
    g = json.load(open(os.path.join(GOLDEN, "cube_corners.json")))
    a = g["a"]
    K = np.array([[sx * a, sy * a, sz * a] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)])
    A, R, G = oracle.forces(K, one_cell())
    sign = np.sign(K)
    np.testing.assert_allclose(R, sign * g["R_component"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(A, sign * g["A_component"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(G, A - R, rtol=0, atol=0)
    F, Fa, Fr = oracle.energy(K, one_cell())
    assert Fa == pytest.approx(g["Fa"], abs=1e-15)
    assert Fr == pytest.approx(g["Fr"], abs=1e-15)
    assert F == pytest.approx(g["Fa"] - g["Fr"], abs=1e-15)


def test_two_samples_closed_form():
    """N = 2: R_1 = (1/2) u = -R_2, u the unit vector from K_2 to K_1 (1/N = 1/2);
    a one-cell density at c: A_i = (K_i - c)/|K_i - c|;
    F^r = (1/(2*4)) * 2 d = d/4, F^a = (|K_1 - c| + |K_2 - c|)/2."""
    rng = np.random.default_rng(3)
    K = rng.uniform(-0.5, 0.5, size=(2, 3))
    grid = one_cell(0.1, 0.3)               # the only cell centre is (0.2, 0.2, 0.2)
    c = np.array([0.2, 0.2, 0.2])
    A, R, G = oracle.forces(K, grid)
    d = K[0] - K[1]
    u = d / np.linalg.norm(d)
    np.testing.assert_allclose(R[0], 0.5 * u, atol=1e-15)
    np.testing.assert_allclose(R[1], -0.5 * u, atol=1e-15)
    for i in range(2):
        v = K[i] - c
        np.testing.assert_allclose(A[i], v / np.linalg.norm(v), atol=1e-15)
    F, Fa, Fr = oracle.energy(K, grid)
    assert Fr == pytest.approx(np.linalg.norm(d) / 4, abs=1e-16)
    assert Fa == pytest.approx(0.5 * sum(np.linalg.norm(K[i] - c) for i in range(2)), abs=1e-16)


def test_delta_density_on_non_cubic_grid():
    """A density with two non-zero cells on a 5 x 3 x 4 grid: the attraction is
    the rho-weighted sum of the two unit vectors; pins the cell-centre
    coordinates lo + (q + 1/2)(hi - lo)/n and the [nz][ny][nx] layout."""
    nx, ny, nz = 5, 3, 4
    rho = np.zeros((nz, ny, nx), np.float32)
    rho[2, 1, 3] = 0.25                    # ix=3, iy=1, iz=2
    rho[0, 2, 1] = 0.75                    # ix=1, iy=2, iz=0
    grid = inputs.Grid((nx, ny, nz), -0.5, 0.5, rho)
    x1 = np.array([-0.5 + 3.5 / 5, -0.5 + 1.5 / 3, -0.5 + 2.5 / 4])
    x2 = np.array([-0.5 + 1.5 / 5, -0.5 + 2.5 / 3, -0.5 + 0.5 / 4])
    K = np.random.default_rng(5).uniform(-0.5, 0.5, size=(7, 3))
    A, _, _ = oracle.forces(K, grid)
    for i in range(7):
        e1 = (K[i] - x1) / np.linalg.norm(K[i] - x1)
        e2 = (K[i] - x2) / np.linalg.norm(K[i] - x2)
        np.testing.assert_allclose(A[i], 0.25 * e1 + 0.75 * e2, atol=1e-15)
    _, Fa, _ = oracle.energy(K, grid)
    ref = np.mean([0.25 * np.linalg.norm(k - x1) + 0.75 * np.linalg.norm(k - x2) for k in K])
    assert Fa == pytest.approx(ref, abs=1e-15)


def test_far_field_attraction():
    """Far from the grid, A -> (k - c)/|k - c| with c = sum_q rho_q x_q, the error
    being O((grid radius / distance)^2)."""
    grid = random_grid((6, 5, 4), seed=1)
    nx, ny, nz = grid.n
    xs = inputs.cell_centres(nx); ys = inputs.cell_centres(ny); zs = inputs.cell_centres(nz)
    rho = grid.rho.astype(np.float64)
    c = np.array([(rho.sum(axis=(0, 1)) * xs).sum(), (rho.sum(axis=(0, 2)) * ys).sum(),
                  (rho.sum(axis=(1, 2)) * zs).sum()])
    dirs = np.random.default_rng(2).normal(size=(5, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    for dist, tol in ((1e2, 1e-4), (1e3, 1e-6)):
        K = dirs * dist
        A, _, _ = oracle.forces(K, grid)
        ref = (K - c) / np.linalg.norm(K - c, axis=1, keepdims=True)
        assert np.abs(A - ref).max() < tol


@pytest.mark.parametrize("n", [8, 7, 32])
def test_symmetric_density_zero_attraction_at_centre(n):
    """A density symmetric under x -> -x attracts nothing at the origin (odd n
    puts a grid point on the origin: the zero-distance term is skipped)."""
    grid = inputs.density_inverse_power(n, 2.0) if n != 7 else inputs.density_gaussian(7, 0.2, 0.01)
    K = np.zeros((3, 3))
    K[1] = [0.3, -0.2, 0.1]
    K[2] = [-0.3, 0.2, -0.1]
    A, R, G = oracle.forces(K, grid)
    assert np.abs(A[0]).max() < 1e-15
    # Mirror symmetry: A(-k) = -A(k).
    np.testing.assert_allclose(A[2], -A[1], atol=1e-15)


def test_repulsion_net_force_zero():
    """The pair terms are antisymmetric, so sum_i R_i = 0."""
    p = inputs.make_problem("tiny")
    _, R, _ = oracle.forces(p.K, p.grid)
    scale = np.abs(R).sum()
    assert np.abs(R.sum(axis=0)).max() < 1e-14 * scale


def test_translation_covariance():
    """R depends only on differences; A is unchanged when samples and grid
    move together."""
    grid = random_grid((4, 3, 5), seed=7)
    K = np.random.default_rng(8).uniform(-0.5, 0.5, size=(40, 3))
    A0, R0, _ = oracle.forces(K, grid)
    t = 0.125                                # exact binary shift
    g2 = inputs.Grid(grid.n, grid.lo + t, grid.hi + t, grid.rho)
    A1, R1, _ = oracle.forces(K + t, g2)
    np.testing.assert_allclose(R1, R0, atol=1e-14)
    np.testing.assert_allclose(A1, A0, atol=1e-14)


def test_axis_permutation_covariance():
    """Permuting the coordinate axes of samples and density permutes A and R;
    a transposed density index would break this."""
    rng = np.random.default_rng(9)
    n = 6
    rho = rng.uniform(0.1, 1.0, size=(n, n, n))
    rho = (rho / rho.sum()).astype(np.float32)
    grid = inputs.Grid((n, n, n), -0.5, 0.5, rho)
    K = rng.uniform(-0.5, 0.5, size=(30, 3))
    A0, R0, _ = oracle.forces(K, grid)
    # new coords (x', y', z') = (y, z, x): rho'[z', y', x'] = rho[z=y', y=x', x=z'].
    Kp = K[:, [1, 2, 0]]
    rhop = np.ascontiguousarray(np.transpose(rho, (2, 0, 1)))
    # check the index map on one entry: rho'[a, b, c] == rho[b, c, a]
    assert rhop[1, 2, 3] == rho[2, 3, 1]
    A1, R1, _ = oracle.forces(Kp, inputs.Grid((n, n, n), -0.5, 0.5, rhop))
    np.testing.assert_allclose(A1, A0[:, [1, 2, 0]], atol=1e-14)
    np.testing.assert_allclose(R1, R0[:, [1, 2, 0]], atol=1e-14)


def test_gradient_matches_central_differences_of_energy():
    """G_i / N equals the central difference of F = F^a - F^r (h = 1e-5)."""
    rng = np.random.default_rng(11)
    grid = random_grid((6, 5, 7), seed=12)
    N = 96
    K = rng.uniform(-0.45, 0.45, size=(N, 3))
    _, _, G = oracle.forces(K, grid)
    h = 1e-5
    for _ in range(24):
        i, c = int(rng.integers(N)), int(rng.integers(3))
        Kp = K.copy(); Kp[i, c] += h
        Km = K.copy(); Km[i, c] -= h
        fd = (oracle.energy(Kp, grid)[0] - oracle.energy(Km, grid)[0]) / (2 * h)
        assert fd == pytest.approx(G[i, c] / N, rel=2e-6, abs=1e-10)


def test_gradient_matches_high_precision_derivative():
    """mpmath (40 digits) differentiates the energy definition numerically;
    the oracle's G/N must agree to ~1e-12 and its energy to ~1e-15."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    rng = np.random.default_rng(13)
    grid = random_grid((3, 2, 2), seed=14, lo=-0.4, hi=0.6)
    nx, ny, nz = grid.n
    N = 6
    K = rng.uniform(-0.5, 0.5, size=(N, 3))
    pts = []
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                x = [mp.mpf(-0.4) + (q + mp.mpf(0.5)) * (mp.mpf(0.6) - mp.mpf(-0.4)) / n
                     for q, n in ((ix, nx), (iy, ny), (iz, nz))]
                pts.append((x, mp.mpf(float(grid.rho[iz, iy, ix]))))

    def dist(a, b):
        return mp.sqrt(sum((a[c] - b[c]) ** 2 for c in range(3)))

    def F(P):
        fa = sum(w * dist(p, x) for p in P for (x, w) in pts) / N
        fr = sum(dist(P[i], P[j]) for i in range(N) for j in range(N) if i != j) / (2 * N * N)
        return fa - fr

    P0 = [[mp.mpf(float(v)) for v in row] for row in K]
    F0 = F(P0)
    assert float(F0) == pytest.approx(oracle.energy(K, grid)[0], rel=1e-14)
    _, _, G = oracle.forces(K, grid)
    for i in range(N):
        for c in range(3):
            def f(t, i=i, c=c):
                P = [row[:] for row in P0]
                P[i][c] = t
                return F(P)
            d = mp.diff(f, P0[i][c])
            assert G[i, c] / N == pytest.approx(float(d), rel=1e-12, abs=1e-15)


def test_targets_subset_matches_full():
    p = inputs.make_problem("tiny")
    idx = np.array([0, 5, 1023, 17, 5])
    A, R, G = oracle.forces(p.K, p.grid)
    A2, R2, G2 = oracle.forces(p.K, p.grid, targets=idx)
    np.testing.assert_array_equal(G2, G[idx])
    np.testing.assert_array_equal(R2, R[idx])


def test_coincident_samples_contribute_nothing():
    """Two samples at the same position: the zero-distance pair is skipped
    (minimum-norm subgradient), the rest is the N = 3 closed form."""
    K = np.array([[0.1, 0.2, 0.3], [0.1, 0.2, 0.3], [-0.2, 0.0, 0.1]])
    _, R, _ = oracle.forces(K, one_cell())
    u = (K[0] - K[2]) / np.linalg.norm(K[0] - K[2])
    np.testing.assert_allclose(R[0], u / 3, atol=1e-16)
    np.testing.assert_allclose(R[1], u / 3, atol=1e-16)
    np.testing.assert_allclose(R[2], -2 * u / 3, atol=1e-16)


def test_invalid_arguments_rejected():
    with pytest.raises(ValueError):
        oracle.forces(np.zeros((4, 3)), one_cell(), targets=[0, 9])
    with pytest.raises(ValueError):
        oracle.forces(np.zeros((4, 3)), inputs.Grid((2, 1, 1), 0.5, -0.5, np.ones((1, 1, 2), np.float32)))


def test_attraction_at_points_matches_forces_and_closed_form():
    """attraction_at evaluates the same attraction as forces (and its
    per-target energy sum) at arbitrary points; at a point far from a
    one-cell density it is the unit vector and the distance."""
    p = inputs.make_problem("tiny")
    idx = np.array([0, 3, 511, 1023])
    A0, _, _, ea, _ = oracle.forces(p.K, p.grid, targets=idx, energies=True)
    A, phi = oracle.attraction_at(p.K[idx], p.grid)
    np.testing.assert_array_equal(A, A0)
    np.testing.assert_array_equal(phi, ea)
    pts = np.array([[0.3, -0.1, 0.2], [0.0, 0.0, 0.0]])
    A1, phi1 = oracle.attraction_at(pts, one_cell(0.0, 0.2))   # cell centre (0.1, 0.1, 0.1)
    d = pts - 0.1
    np.testing.assert_allclose(A1, d / np.linalg.norm(d, axis=1, keepdims=True), atol=1e-15)
    np.testing.assert_allclose(phi1, np.linalg.norm(d, axis=1), atol=1e-15)


# --- regularised kernel H(r) = sqrt(r^2 + eps^2) (Sec. II-C, choice of step size)

def test_regularised_two_samples_closed_form():
    """N = 2 and one density cell: R_1 = (1/2) e / sqrt(|e|^2 + eps^2) = -R_2,
    A_i = d_i / sqrt(|d_i|^2 + eps^2), F^r = 2 sqrt(|e|^2 + eps^2) / (2 N^2)."""
    eps = 0.07
    K = np.array([[0.1, -0.2, 0.05], [-0.15, 0.1, 0.2]])
    grid = one_cell(0.0, 0.2)                    # cell centre (0.1, 0.1, 0.1)
    A, R, G = oracle.forces(K, grid, eps=eps)
    e = K[0] - K[1]
    re = math.sqrt(e @ e + eps * eps)
    np.testing.assert_allclose(R[0], 0.5 * e / re, rtol=0, atol=1e-16)
    np.testing.assert_allclose(R[1], -0.5 * e / re, rtol=0, atol=1e-16)
    d = K - 0.1
    rd = np.sqrt((d * d).sum(1) + eps * eps)
    np.testing.assert_allclose(A, d / rd[:, None], rtol=0, atol=1e-16)
    F, Fa, Fr = oracle.energy(K, grid, eps=eps)
    assert Fr == pytest.approx(2 * re / 8, rel=1e-15)
    assert Fa == pytest.approx(rd.sum() / 2, rel=1e-15)


def test_regularised_coincident_samples_and_grid_point():
    """With eps > 0 nothing is singular: two coincident samples repel with
    zero force but add eps each to the directed distance sums (F^r = 2 eps /
    (2 N^2) for N = 2), and a sample on a grid point adds rho eps to F^a."""
    eps = 0.01
    grid = one_cell(0.0, 0.2)
    K = np.array([[0.1, 0.1, 0.1], [0.1, 0.1, 0.1]])
    A, R, G = oracle.forces(K, grid, eps=eps)
    np.testing.assert_array_equal(R, 0.0)
    np.testing.assert_array_equal(A, 0.0)
    F, Fa, Fr = oracle.energy(K, grid, eps=eps)
    assert Fr == pytest.approx(2 * eps / 8, rel=1e-15)
    assert Fa == pytest.approx(eps, rel=1e-15)


def test_regularised_gradient_matches_central_differences():
    """G / N is the derivative of the regularised energy, also at a pair of
    coincident samples and at samples on grid points, where the plain norm
    has a kink (h = 1e-6 against eps = 0.02: the energy is smooth there)."""
    rng = np.random.default_rng(31)
    grid = random_grid((4, 5, 3), seed=32)
    eps = 0.02
    N = 40
    K = rng.uniform(-0.45, 0.45, size=(N, 3))
    K[1] = K[0]                                  # coincident pair
    K[2] = [-0.5 + 0.5 / 4, -0.5 + 1.5 / 5, -0.5 + 2.5 / 3]   # a grid point
    _, _, G = oracle.forces(K, grid, eps=eps)
    h = 1e-6
    for i, c in [(0, 0), (1, 2), (2, 1), (2, 0)] + [(int(rng.integers(N)), int(rng.integers(3)))
                                                    for _ in range(12)]:
        Kp = K.copy(); Kp[i, c] += h
        Km = K.copy(); Km[i, c] -= h
        fd = (oracle.energy(Kp, grid, eps=eps)[0] - oracle.energy(Km, grid, eps=eps)[0]) / (2 * h)
        assert fd == pytest.approx(G[i, c] / N, rel=1e-6, abs=1e-10)


def test_regularised_tends_to_plain_norm():
    """eps -> 0 recovers the plain kernel (no coincident points): the
    difference of each unit-vector term is O(eps^2 / r^2)."""
    p = inputs.make_problem("tiny")
    A0, R0, G0 = oracle.forces(p.K, p.grid)
    A1, R1, G1 = oracle.forces(p.K, p.grid, eps=1e-7)
    assert np.abs(G1 - G0).max() < 1e-6
    F0 = oracle.energy(p.K, p.grid)
    F1 = oracle.energy(p.K, p.grid, eps=1e-7)
    assert F1[0] == pytest.approx(F0[0], rel=1e-9)
    # and eps changes the result visibly when it is not small
    A2, _, _ = oracle.forces(p.K, p.grid, eps=0.05)
    assert np.abs(A2 - A0).max() > 1e-3


def test_energy_terms_pins():
    """energy_terms (the terms of F that contain one sample, with the sample
    moved): closed form for N = 2 and one density point; at the samples' own
    positions the per-target sums of forces(); summed over the samples, F^a
    and twice F^r (eq. global_minimization); its central differences times N
    equal G (the repulsion's double sum counts each pair twice, a plausible
    factor-2 mistake)."""
    grid = one_cell(0.1, 0.3)
    K = np.array([[0.3, -0.1, 0.2], [-0.2, 0.25, 0.0]])
    p = np.array([[0.05, 0.1, -0.3]])
    ea, er = oracle.energy_terms(K, grid, [0], p)
    assert ea[0] == pytest.approx(np.linalg.norm(p[0] - 0.2), abs=1e-15)
    assert er[0] == pytest.approx(np.linalg.norm(p[0] - K[1]), abs=1e-15)

    rng = np.random.default_rng(31)
    K = rng.uniform(-0.5, 0.5, size=(300, 3))
    grid = random_grid((5, 7, 6), 32)
    idx = np.arange(300)
    ea, er = oracle.energy_terms(K, grid, idx, K)
    _, _, _, ea0, er0 = oracle.forces(K, grid, energies=True)
    np.testing.assert_array_equal(ea, ea0)
    np.testing.assert_array_equal(er, er0)
    _, Fa, Fr = oracle.energy(K, grid)
    assert ea.sum() / 300 == pytest.approx(Fa, rel=1e-14)
    assert er.sum() / (2 * 300 ** 2) == pytest.approx(Fr, rel=1e-14)

    N, h = 300, 1e-5
    _, _, G = oracle.forces(K, grid)
    tgt = np.array([3, 77, 150, 299])
    for c in range(3):
        pp, pm = K[tgt].copy(), K[tgt].copy()
        pp[:, c] += h
        pm[:, c] -= h
        eap, erp = oracle.energy_terms(K, grid, tgt, pp)
        eam, erm = oracle.energy_terms(K, grid, tgt, pm)
        fd = ((eap / N - erp / N ** 2) - (eam / N - erm / N ** 2)) / (2 * h) * N
        np.testing.assert_allclose(fd, G[tgt, c], rtol=0, atol=1e-7)
    with pytest.raises(ValueError):
        oracle.energy_terms(K, grid, [300], K[:1])
