"""Seeded synthetic inputs for the SPARKLING hot path.

This module is shared by the FP64 oracle (``oracle/``), the tests and the
benchmark.  It only *draws* inputs: sample positions, target densities on a
Cartesian grid and per-trajectory constants.  It holds none of the method's
arithmetic (no attraction, repulsion, energy or projection code).

Shapes follow the paper's workloads (arxiv 2108.02991):

* samples live in [-1/2, 1/2]^3, the paper's Omega = [-1, 1]^3 (Sec. II-A)
  scaled by 1/2;
* a pattern is N_c shots x N_s samples, stored shot after shot, giving an
  ``[N, 3]`` array with N = N_c * N_s (Sec. II-A, eq. ktraj);
* initial trajectories are radial spokes through the k-space centre with an
  optional zero-mean uniform perturbation (Sec. III-A.2, Fig. add_perturbation);
* target densities are radially symmetric with a central plateau and an
  inverse-power decay (Sec. III-A.1, eq. target_distribution), or Gaussian
  with a floor;
* the density grid is cell-centred: along each axis of n cells on [lo, hi]
  the points are lo + (q + 1/2) (hi - lo) / n, q = 0 .. n-1.  The array is
  C-ordered ``[nz, ny, nx]`` (x fastest) and normalised to sum 1.

All randomness comes from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

__all__ = [
    "Grid", "Proj", "Problem", "uniform_points", "hemisphere_directions",
    "radial_spokes", "perturb_uniform", "cell_centres", "density_inverse_power",
    "density_gaussian", "make_problem", "make_batched", "CONFIG_NAMES",
]

CONFIG_NAMES = ("tiny", "small", "medium", "diff", "batched", "hr")


@dataclasses.dataclass
class Grid:
    """Cell-centred density grid on [lo, hi]^3; rho is float32 [nz, ny, nx]."""
    n: tuple            # (nx, ny, nz)
    lo: float
    hi: float
    rho: np.ndarray


@dataclasses.dataclass
class Proj:
    """Constraint-set parameters of one trajectory (eq. constraints)."""
    alpha: float
    beta: float
    box: float = 0.5
    pin_index: int = -1
    pin: tuple = (0.0, 0.0, 0.0)
    n_iter: int = 100
    tol: float = 0.0
    margin: float = 0.0


@dataclasses.dataclass
class Problem:
    name: str
    K: np.ndarray       # [N, 3], float32 or float64
    Nc: int
    Ns: int
    grid: Grid
    proj: Proj
    eta: float
    iterations: int
    recipe: str

    @property
    def N(self) -> int:
        return int(self.K.shape[0])


def uniform_points(n: int, seed: int = 0, dtype=np.float64) -> np.ndarray:
    """n points uniform in [-1/2, 1/2]^3."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-0.5, 0.5, size=(n, 3)).astype(dtype)


def hemisphere_directions(nc: int) -> np.ndarray:
    """nc unit vectors spread over the upper hemisphere by a golden-angle
    (Fibonacci) spiral.  A full-diameter spoke along u also covers -u, so a
    hemisphere of directions covers the sphere."""
    i = np.arange(nc, dtype=np.float64)
    z = (i + 0.5) / nc
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    rxy = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([rxy * np.cos(phi), rxy * np.sin(phi), z], axis=1)


def radial_spokes(nc: int, ns: int, radius: float, jitter: float = 0.0,
                  seed: int = 0, dtype=np.float64) -> np.ndarray:
    """nc straight spokes through the centre, ns samples each, from -radius*u
    to +radius*u, plus optional N(0, jitter^2) noise per coordinate.
    Returned as [nc*ns, 3], shot after shot."""
    u = hemisphere_directions(nc)
    t = radius * (2.0 * np.arange(ns, dtype=np.float64) / max(ns - 1, 1) - 1.0)
    K = u[:, None, :] * t[None, :, None]
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        K = K + rng.normal(0.0, jitter, size=K.shape)
    K = np.clip(K, -0.5, 0.5)
    return K.reshape(nc * ns, 3).astype(dtype)


def perturb_uniform(K: np.ndarray, amplitude: float, seed: int = 0) -> np.ndarray:
    """Add zero-mean uniform noise in [-amplitude, amplitude] to every
    coordinate and clip back into [-1/2, 1/2]."""
    rng = np.random.default_rng(seed)
    out = K.astype(np.float64) + rng.uniform(-amplitude, amplitude, size=K.shape)
    return np.clip(out, -0.5, 0.5).astype(K.dtype)


def cell_centres(n: int, lo: float = -0.5, hi: float = 0.5) -> np.ndarray:
    """Coordinates of the n cell centres of [lo, hi] (float64)."""
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * ((hi - lo) / n)


def _radius_grid(n: int) -> np.ndarray:
    c = cell_centres(n)
    return np.sqrt(c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2)


def _normalised(rho: np.ndarray) -> np.ndarray:
    rho = rho / rho.sum(dtype=np.float64)
    return np.ascontiguousarray(rho.astype(np.float32))


def density_inverse_power(n: int, power: float, r0: Optional[float] = None) -> Grid:
    """rho(x) proportional to 1 / max(|x|, r0)^power on an n^3 cell-centred
    grid over [-1/2, 1/2]^3 (plateau of radius r0, then inverse-power decay);
    r0 defaults to 1/n."""
    r0 = 1.0 / n if r0 is None else r0
    rho = 1.0 / np.maximum(_radius_grid(n), r0) ** power
    return Grid((n, n, n), -0.5, 0.5, _normalised(rho))


def density_gaussian(n: int, sigma: float, floor: float = 0.0) -> Grid:
    """rho(x) proportional to exp(-|x|^2 / (2 sigma^2)) + floor on n^3 cells."""
    r = _radius_grid(n)
    rho = np.exp(-(r * r) / (2.0 * sigma * sigma)) + floor
    return Grid((n, n, n), -0.5, 0.5, _normalised(rho))


def _alpha_beta(ns: int):
    # Per-step constraints in [-1/2,1/2] units used by every synthetic config.
    return 1.0 / (2.0 * ns), 1.0 / (8.0 * ns * ns)


def make_problem(name: str, seed: int = 0) -> Problem:
    """Build one of the synthetic workloads: tiny, medium, diff or hr."""
    if name == "tiny":
        nc, ns = 16, 64
        a, b = _alpha_beta(ns)
        K = uniform_points(nc * ns, seed, np.float64)
        grid = density_inverse_power(32, 2.0)
        return Problem(name, K, nc, ns, grid, Proj(a, b), 1.0 / (nc * ns), 1,
                       "16x64 uniform in [-1/2,1/2]^3 (f64); rho ~ 1/max(|x|,1/32)^2 on 32^3")
    if name in ("small", "medium", "diff", "hr"):
        if name == "small":
            # a representative case small enough for detailed profiler captures
            nc, ns, dtype = 64, 1024, np.float32
            grid = density_inverse_power(64, 2.0)
            iters = 1
        elif name == "medium":
            nc, ns, dtype = 512, 512, np.float32
            grid = density_gaussian(128, 0.15, 0.05)
            iters = 10
        elif name == "diff":
            nc, ns, dtype = 2048, 512, np.float32
            grid = density_inverse_power(192, 1.5)
            iters = 1
        else:
            nc, ns, dtype = 4096, 2560, np.float32
            grid = density_inverse_power(256, 2.0)
            iters = 1
        a, b = _alpha_beta(ns)
        radius = 0.95 * a * (ns - 1) / 2.0
        K = radial_spokes(nc, ns, radius, jitter=1e-3, seed=seed, dtype=np.float64)
        if name == "hr":
            K = perturb_uniform(K, 0.375, seed=seed + 1)
        K = K.astype(dtype)
        proj = Proj(a, b, pin_index=ns // 2, pin=(0.0, 0.0, 0.0))
        recipe = (f"{nc}x{ns} golden-spiral radial spokes, radius {radius:.6f}, "
                  f"N(0,1e-3^2) jitter" + (", uniform +-0.375 perturbation" if name == "hr" else "")
                  + f"; {grid.n[0]}^3 density")
        return Problem(name, K, nc, ns, grid, proj, 1.0 / (nc * ns), iters, recipe)
    raise ValueError(f"unknown problem {name!r}")


def make_batched(n_traj: int = 64, ns: int = 512, grid_n: int = 64, seed: int = 0,
                 min_shots: int = 32, max_shots: int = 512):
    """Batch of independent trajectories of uneven size: N_b = ns * U{min..max}
    shots, spokes with their own seed, a Gaussian density per trajectory with
    sigma_b ~ U[0.1, 0.3], alpha_b, beta_b scaled by U[0.5, 1.5]."""
    rng = np.random.default_rng(seed)
    shots = rng.integers(min_shots, max_shots + 1, size=n_traj)
    sig = rng.uniform(0.1, 0.3, size=n_traj)
    sa = rng.uniform(0.5, 1.5, size=n_traj)
    sb = rng.uniform(0.5, 1.5, size=n_traj)
    probs = []
    a0, b0 = _alpha_beta(ns)
    for b in range(n_traj):
        nc = int(shots[b])
        a = a0 * sa[b]
        radius = 0.95 * a * (ns - 1) / 2.0
        K = radial_spokes(nc, ns, radius, jitter=1e-3, seed=seed + 1000 + b,
                          dtype=np.float64).astype(np.float32)
        grid = density_gaussian(grid_n, float(sig[b]))
        probs.append(Problem(f"batched[{b}]", K, nc, ns, grid,
                             Proj(a, b0 * sb[b]), 1.0 / (nc * ns), 1,
                             f"spokes seed {seed + 1000 + b}, gaussian sigma {sig[b]:.4f}"))
    return probs
