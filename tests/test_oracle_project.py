"""Pins of the oracle's per-shot projection (eq. constraints, Sec. II-D,
Suppl. Sec. I) against closed forms, a general-purpose solver (scipy SLSQP)
and the properties every Euclidean projection onto a convex set has."""
import math

import numpy as np
import pytest

import oracle

INF = float("inf")


def smooth_shot(ns, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    t = np.linspace(0, 1, ns)[:, None]
    a = rng.normal(size=(3, 3))
    return scale * np.tanh(np.hstack([np.sin(2 * t * a[0, c] + a[1, c]) for c in range(3)]) * a[2])


def test_box_only_is_clipping():
    """alpha = beta = inf leaves only the box: the projection is clipping."""
    K = np.random.default_rng(0).uniform(-0.8, 0.8, size=(4 * 16, 3))
    s = oracle.project(K, 4, 16, INF, INF, box=0.5, n_iter=7)
    np.testing.assert_array_equal(s, np.clip(K, -0.5, 0.5))


def test_two_samples_amplitude_closed_form():
    """N_s = 2 with only the amplitude bound: s = m -/+ (alpha/2) u, the two
    samples pulled symmetrically towards their midpoint m."""
    rng = np.random.default_rng(1)
    K = rng.uniform(-0.2, 0.2, size=(2, 3))
    alpha = 0.05
    s = oracle.project(K, 1, 2, alpha, 1.0, n_iter=2000)
    m = K.mean(axis=0)
    u = (K[1] - K[0]) / np.linalg.norm(K[1] - K[0])
    np.testing.assert_allclose(s[0], m - alpha / 2 * u, atol=1e-12)
    np.testing.assert_allclose(s[1], m + alpha / 2 * u, atol=1e-12)


def test_three_samples_slew_closed_form():
    """N_s = 3 with only the slew bound: with L = [1, -2, 1] (|L|^2 = 6),
    s = k - L^T (L k)(1 - beta/|L k|)/6."""
    rng = np.random.default_rng(2)
    K = rng.uniform(-0.2, 0.2, size=(3, 3))
    beta = 0.01
    s = oracle.project(K, 1, 3, INF, beta, n_iter=4000)
    L = np.array([1.0, -2.0, 1.0])
    w = L @ K
    ref = K - np.outer(L, w) * (1 - beta / np.linalg.norm(w)) / 6
    np.testing.assert_allclose(s, ref, atol=1e-12)


def fista_scalar(kind, c, rad, n):
    """The dual FISTA recursion written out for a one-dimensional motion
    (x component only).  kind 'amp': N_s = 2, k = (0, c), s(q) = (q, c - q),
    D1 s = c - 2q.  kind 'slew': N_s = 3, k = (0, c, 0),
    s(q) = (-q, c + 2q, -q), D2 s = -2c - 6q.  tau = 1/20."""
    tau = 1.0 / 20.0
    q = y = 0.0
    t = 1.0
    for _ in range(n):
        ds = (c - 2 * y) if kind == "amp" else (-2 * c - 6 * y)
        z = y + tau * ds
        qn = math.copysign(max(0.0, abs(z) - tau * rad), z)
        tn = 0.5 * (1 + math.sqrt(1 + 4 * t * t))
        y = qn + (t - 1) / tn * (qn - q)
        q, t = qn, tn
    return (q, c - q) if kind == "amp" else (-q, c + 2 * q, -q)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 20, 60])
def test_fista_iterates_one_dimensional(n):
    """Fixed-iteration outputs equal the hand-reduced scalar recursion: pins
    the step 1/20, the momentum schedule, the adjoint signs and that the
    output is s(q), not s(y)."""
    c, alpha = 0.3, 0.01
    K = np.zeros((2, 3)); K[1, 0] = c
    s = oracle.project(K, 1, 2, alpha, 1.0, n_iter=n)
    np.testing.assert_allclose(s[:, 0], fista_scalar("amp", c, alpha, n), rtol=0, atol=1e-15)
    assert np.all(s[:, 1:] == 0)
    c, beta = 0.2, 0.003
    K = np.zeros((3, 3)); K[1, 0] = c
    s = oracle.project(K, 1, 3, INF, beta, n_iter=n)
    np.testing.assert_allclose(s[:, 0], fista_scalar("slew", c, beta, n), rtol=0, atol=1e-15)


def slsqp_projection(k, alpha, beta, box, pin_index=-1, pin=None):
    """Reference projection by scipy's SLSQP on min 1/2|s - k|^2 subject to the
    squared-norm form of the constraints."""
    opt = pytest.importorskip("scipy.optimize")
    ns = k.shape[0]

    def f(x):
        d = x - k.ravel()
        return 0.5 * d @ d, d

    def cons(x):
        s = x.reshape(ns, 3)
        d1 = s[1:] - s[:-1]
        d2 = s[2:] - 2 * s[1:-1] + s[:-2]
        return np.concatenate([alpha ** 2 - (d1 * d1).sum(1), beta ** 2 - (d2 * d2).sum(1)])

    def jac(x):
        s = x.reshape(ns, 3)
        rows = []
        for n in range(ns - 1):
            J = np.zeros((ns, 3)); d = s[n + 1] - s[n]
            J[n + 1] -= 2 * d; J[n] += 2 * d
            rows.append(J.ravel())
        for n in range(ns - 2):
            J = np.zeros((ns, 3)); d = s[n + 2] - 2 * s[n + 1] + s[n]
            J[n + 2] -= 2 * d; J[n + 1] += 4 * d; J[n] -= 2 * d
            rows.append(J.ravel())
        return np.array(rows)

    constraints = [{"type": "ineq", "fun": cons, "jac": jac}]
    if pin_index >= 0:
        def eq(x):
            return x.reshape(ns, 3)[pin_index] - np.asarray(pin)

        def eqj(x):
            J = np.zeros((3, ns * 3))
            for c in range(3):
                J[c, 3 * pin_index + c] = 1.0
            return J
        constraints.append({"type": "eq", "fun": eq, "jac": eqj})
    x0 = np.clip(k.ravel(), -box, box) * 0.5
    res = opt.minimize(f, x0, jac=True, method="SLSQP", bounds=[(-box, box)] * (3 * ns),
                       constraints=constraints, options={"ftol": 1e-15, "maxiter": 2000})
    assert res.success, res.message
    return res.x.reshape(ns, 3)


@pytest.mark.parametrize("seed,pin_index", [(3, -1), (4, -1), (5, 4)])
def test_matches_general_solver(seed, pin_index):
    """Many FISTA iterations reach the projection found by SLSQP, with the
    amplitude, slew, box (and pin) constraints all active."""
    rng = np.random.default_rng(seed)
    ns = 9
    k = rng.uniform(-0.3, 0.3, size=(ns, 3))
    k[2, 1] = 0.62                                  # outside the box
    alpha, beta, box = 0.12, 0.05, 0.5
    pin = (0.01, -0.02, 0.03)
    ref = slsqp_projection(k, alpha, beta, box, pin_index, pin)
    s = oracle.project(k, 1, ns, alpha, beta, box, pin_index=pin_index, pin=pin, n_iter=300000)
    np.testing.assert_allclose(s, ref, atol=2e-7)
    v = oracle.violation(s, 1, ns, alpha, beta, box, pin_index, pin)
    assert v.max() < 1e-7


def test_idempotent_on_feasible_input_bitwise():
    """A strictly feasible shot is a fixed point: the duals stay at zero and
    the output equals the input bit for bit."""
    k = smooth_shot(64, 6, scale=0.2)
    d1 = np.linalg.norm(np.diff(k, axis=0), axis=1).max()
    d2 = np.linalg.norm(np.diff(k, 2, axis=0), axis=1).max()
    s = oracle.project(k, 1, 64, 1.01 * d1, 1.01 * d2, n_iter=50)
    np.testing.assert_array_equal(s, k)


def converged(k, ns, alpha, beta, tol=1e-11):
    s, it = oracle.project(k, k.shape[0] // ns, ns, alpha, beta, n_iter=2_000_000, tol=tol,
                           margin=0.0, check_every=50, return_iters=True)
    return s


def test_converged_mode_certificate():
    """Converged mode stops on a feasibility + duality-gap certificate; the
    answer is within sqrt(2 tol) of SLSQP's and feasible to tol."""
    rng = np.random.default_rng(7)
    ns = 8
    k = rng.uniform(-0.25, 0.25, size=(ns, 3))
    alpha, beta, tol = 0.1, 0.04, 1e-12
    s, it = oracle.project(k, 1, ns, alpha, beta, n_iter=2_000_000, tol=tol, check_every=10,
                           return_iters=True)
    assert it[0] < 2_000_000
    assert oracle.violation(s, 1, ns, alpha, beta).max() <= tol
    ref = slsqp_projection(k, alpha, beta, 0.5)
    assert np.abs(s - ref).max() < math.sqrt(2 * tol) + 1e-7


def test_margin_gives_strict_feasibility():
    """With margin mu the target set is shrunk by (1 - mu): the result is
    strictly inside the requested set."""
    k = np.random.default_rng(8).uniform(-0.25, 0.25, size=(10, 3))
    alpha, beta = 0.1, 0.04
    s = oracle.project(k, 1, 10, alpha, beta, n_iter=2_000_000, tol=1e-9, margin=1e-4)
    d1 = np.linalg.norm(np.diff(s, axis=0), axis=1).max()
    d2 = np.linalg.norm(np.diff(s, 2, axis=0), axis=1).max()
    assert d1 < alpha and d2 < beta


def test_nonexpansive_and_variational_inequality():
    """|P(a) - P(b)| <= |a - b|, and <k - P(k), s - P(k)> <= 0 for feasible s
    (here s = lambda P(k), feasible because the set is convex and holds 0)."""
    rng = np.random.default_rng(9)
    ns, alpha, beta = 12, 0.08, 0.03
    a = rng.uniform(-0.3, 0.3, size=(ns, 3))
    b = a + rng.normal(scale=0.05, size=(ns, 3))
    pa, pb = converged(a, ns, alpha, beta), converged(b, ns, alpha, beta)
    assert np.linalg.norm(pa - pb) <= np.linalg.norm(a - b) * (1 + 1e-6)
    for lam in (0.0, 0.3, 0.9, 0.999):
        sv = lam * pa
        assert np.sum((a - pa) * (sv - pa)) <= 1e-8
    # Projecting the projection changes nothing (up to the certificate tolerance).
    np.testing.assert_allclose(converged(pa, ns, alpha, beta), pa, atol=1e-6)


def test_shots_are_independent():
    """Projecting a pattern is projecting each shot (Suppl. Sec. I)."""
    rng = np.random.default_rng(10)
    ns, nc = 16, 5
    K = rng.uniform(-0.3, 0.3, size=(nc * ns, 3))
    s = oracle.project(K, nc, ns, 0.05, 0.01, n_iter=37)
    for c in range(nc):
        sc = oracle.project(K[c * ns:(c + 1) * ns], 1, ns, 0.05, 0.01, n_iter=37)
        np.testing.assert_array_equal(s[c * ns:(c + 1) * ns], sc)


def test_single_sample_shot():
    """N_s = 1: no difference constraints, only box and pin."""
    K = np.array([[0.7, -0.1, 0.2], [0.1, 0.2, -0.9]])
    s = oracle.project(K, 2, 1, 0.01, 0.01, n_iter=5)
    np.testing.assert_array_equal(s, np.clip(K, -0.5, 0.5))
    s = oracle.project(K, 2, 1, 0.01, 0.01, pin_index=0, pin=(0.0, 0.1, 0.0), n_iter=5)
    np.testing.assert_array_equal(s, [[0.0, 0.1, 0.0]] * 2)


def test_step_descends_energy():
    """With the constraints inactive, a small step K - eta G lowers F
    (G = N dF/dK is an ascent direction)."""
    import inputs
    rng = np.random.default_rng(11)
    grid = inputs.density_inverse_power(8, 2.0)
    K = rng.uniform(-0.4, 0.4, size=(4 * 8, 3))
    F0 = oracle.energy(K, grid)[0]
    K1 = oracle.step(K, 4, 8, grid, eta=1e-3, alpha=INF, beta=INF, n_iter=3)
    _, _, G = oracle.forces(K, grid)
    np.testing.assert_allclose(K1, K - 1e-3 * G, atol=1e-16)
    assert oracle.energy(K1, grid)[0] < F0
