"""CPU checks of the fast-repulsion pieces: pins of the oracle's exact
short/long split of the repulsion kernel (oracle.repulsion_split), and the
self-checks of the diagnostic mesh restatement (tests/mesh_reference.py:
the cubic B-spline window, and its long-range sum against the oracle's exact
long-range sum)."""
import math

import numpy as np
import pytest

import inputs
import oracle
import mesh_reference as p3m


def test_bspline_window():
    """Textbook values of the cubic cardinal B-spline, its symmetry, and the
    partition of unity of the four weights of any position."""
    assert p3m.bspline4(np.array([2.0]))[0] == pytest.approx(2.0 / 3.0, abs=1e-15)
    assert p3m.bspline4(np.array([1.0]))[0] == pytest.approx(1.0 / 6.0, abs=1e-15)
    assert p3m.bspline4(np.array([3.0]))[0] == pytest.approx(1.0 / 6.0, abs=1e-15)
    t = np.linspace(0, 4, 97)
    np.testing.assert_allclose(p3m.bspline4(t), p3m.bspline4(4 - t), atol=1e-15)
    u = np.random.default_rng(1).uniform(2, 30, size=1000)
    n0 = np.floor(u) - 1
    tot = sum(p3m.bspline4(u - (n0 + k) + 2) for k in range(4))
    np.testing.assert_allclose(tot, 1.0, atol=1e-14)


@pytest.mark.parametrize("eps", [0.0, 0.02])
def test_split_adds_up_to_the_repulsion(eps):
    """Short (no cut) + long parts = the oracle's repulsion and distance
    sums, for any split width; the short part cut at 4 sigma differs from
    the uncut one by less than the erfc(4) tail."""
    g = inputs.density_gaussian(4, 0.2)
    K = np.random.default_rng(2).uniform(-0.45, 0.45, size=(400, 3))
    K[1] = K[0]                                   # a coincident pair
    N = K.shape[0]
    _, R, _, _, er = oracle.forces(K, g, energies=True, eps=eps)
    for sigma in (0.01, 0.1, 0.7):
        S, L, eS, eL = oracle.repulsion_split(K, sigma, eps=eps)
        np.testing.assert_allclose(S + L, N * R, rtol=0, atol=1e-12)
        np.testing.assert_allclose(eS + eL, er, rtol=1e-13)
    sigma = 0.05
    S, _, eS, _ = oracle.repulsion_split(K, sigma, eps=eps)
    Sc, _, eSc, _ = oracle.repulsion_split(K, sigma, rc=4 * sigma, eps=eps)
    tail = N * math.erfc(4.0)
    assert np.abs(Sc - S).max() <= tail
    assert np.abs(eSc - eS).max() <= tail * 4 * sigma


@pytest.mark.parametrize("eps,sig_cells", [(0.0, 2.5), (0.02, 2.5), (0.0, 3.0)])
def test_mesh_long_range_matches_exact_sum(eps, sig_cells):
    """The particle-mesh long-range sum (24 mesh cells, B-spline window,
    tapered deconvolved kernel) matches the exact long-range sum: the force
    to about 1e-6 (relative L2, falling with sigma / h), the potential to
    about 1e-5 of its largest value (the mesh adds the self term g(0); the
    error of the linearly growing potential does not depend on sigma and
    falls like h^4.5: 1.1e-5 at 24 cells, 3e-6 at 32)."""
    spec = p3m.MeshSpec(n_cells=24, sigma=sig_cells / 24)
    K = np.random.default_rng(3).uniform(-0.5, 0.5, size=(600, 3))
    Lm, eLm = p3m.mesh_long(K, spec, eps)
    _, L, _, eL = oracle.repulsion_split(K, spec.sigma, eps=eps)
    err = np.linalg.norm(Lm - L) / np.linalg.norm(L)
    assert err < 2e-6, err
    perr = np.abs(eLm - p3m.self_potential(spec, eps) - eL).max() / np.abs(eL).max()
    assert perr < 2e-5, perr


def test_mesh_rejects_samples_outside():
    spec = p3m.MeshSpec(n_cells=8, sigma=0.3)
    with pytest.raises(ValueError):
        p3m.mesh_long(np.array([[0.0, 0.0, 0.9], [0.1, 0.1, 0.1]]), spec)
