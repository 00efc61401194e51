"""Particle-mesh long-range part of the repulsion, plain NumPy (FP64): a
diagnostic restatement of the library's own mesh design.

NOT AN ORACLE.  It follows the same steps as the library's mesh summation
(window, taper, guard cells, deconvolution), so a mistake in that design
would be shared by both; no test's pass or fail rests on it.  The mesh
tests gate the library against the exact direct sum (the oracle) within a
stated method-error bound, and print this module's result beside it to help
read a failure.  Only tests/ import it; it shares nothing with the CUDA
library.

The paper evaluates the repulsion with a fast multipole method (Sec. II-C.2)
because the direct sum is O(N^2).  The library's fast repulsion is a
particle-particle particle-mesh (P3M) summation instead: the kernel
d/|d|_eps splits exactly into a short-range part d/r erfc(r/sigma) (summed
directly over close pairs; ``oracle.repulsion_split``) and the smooth
long-range part d/r erf(r/sigma), r = |d|_eps, which this module evaluates
on a mesh in these steps:

1. Mesh: nodes x_n = lo - g h + n h, n = 0..M-1 per axis, h = (hi - lo)/n_cells,
   M = n_cells + 2g (g guard cells).  A sample at mesh coordinate
   u = (x - lo + g h)/h spreads unit charge to the 4 nodes n = floor(u)-1 ..
   floor(u)+2 per axis with weights M4(u - n + 2), M4 the cubic cardinal
   B-spline on [0, 4] (tensor product over the axes).
2. Kernel: the long-range kernel g(x) (3 force components and the potential
   r erf(r/sigma) + sigma/sqrt(pi) exp(-r^2/sigma^2)) is sampled at the
   offsets m h of a periodic box of Lb = 4M points per axis, multiplied by a
   C-infinity taper that is 1 up to radius sqrt(3) M h (every offset two
   mesh nodes can have) and 0 from 2 M h (the box edge), Fourier
   transformed, divided by the squared Fourier transform of the spreading
   window, (prod_a sinc(f_a))^8 (deconvolution; sinc(f) = sin(pi f)/(pi f),
   f in cycles per sample), and transformed back.  The taper makes the
   kernel smooth and compactly supported, so the division does not amplify a
   truncation edge (the free-space convolution idea of Vico, Greengard and
   Ferrando, J. Comput. Phys. 2016).
3. Convolution: the deconvolved kernel at offsets |m_a| < M and the charge
   mesh are convolved cyclically on a box of L = 2M points per axis, which
   equals the linear convolution on the M^3 nodes.
4. Interpolation: each sample gathers the convolved field from the nodes it
   spread to, with the same weights.

The result approximates sum_{j != i} g(k_i - k_j) plus, for the potential,
the self term g(0); its error against the exact sum is measured by the tests.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import erf


@dataclass
class MeshSpec:
    n_cells: int          # mesh cells across [lo, hi]
    sigma: float          # split width (absolute units)
    lo: float = -0.5
    hi: float = 0.5
    guard: int = 4        # guard cells on each side

    @property
    def h(self) -> float:
        return (self.hi - self.lo) / self.n_cells

    @property
    def M(self) -> int:
        return self.n_cells + 2 * self.guard


def bspline4(t):
    """Cubic cardinal B-spline on [0, 4] (zero outside)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros_like(t)
    a = (t >= 0) & (t < 1)
    out[a] = t[a] ** 3 / 6
    b = (t >= 1) & (t < 2)
    tb = t[b]
    out[b] = (-3 * tb ** 3 + 12 * tb ** 2 - 12 * tb + 4) / 6
    c = (t >= 2) & (t < 3)
    tc = t[c]
    out[c] = (3 * tc ** 3 - 24 * tc ** 2 + 60 * tc - 44) / 6
    d = (t >= 3) & (t < 4)
    out[d] = (4 - t[d]) ** 3 / 6
    return out


def spread_weights(K, spec: MeshSpec):
    """Per sample the first node per axis [N, 3] and the weights [N, 3, 4]."""
    u = (np.asarray(K, np.float64) - (spec.lo - spec.guard * spec.h)) / spec.h
    first = np.floor(u).astype(np.int64) - 1
    if first.min() < 0 or first.max() + 3 >= spec.M:
        raise ValueError("a sample lies outside the mesh")
    w = np.stack([bspline4(u - (first + k) + 2) for k in range(4)], axis=-1)
    return first, w


def charges(K, spec: MeshSpec) -> np.ndarray:
    """Charge mesh Q[z][y][x] of unit charges at the samples."""
    first, w = spread_weights(K, spec)
    M = spec.M
    Q = np.zeros((M, M, M))
    for a in range(4):
        for b in range(4):
            for c in range(4):
                np.add.at(Q, (first[:, 2] + c, first[:, 1] + b, first[:, 0] + a),
                          w[:, 0, a] * w[:, 1, b] * w[:, 2, c])
    return Q


def _taper(r, r1, r2):
    t = np.clip((r - r1) / (r2 - r1), 0.0, 1.0)

    def f(x):
        out = np.zeros_like(x)
        pos = x > 0
        out[pos] = np.exp(-1.0 / x[pos])
        return out

    a, b = f(1.0 - t), f(t)
    return a / (a + b)


def kernel_offsets(spec: MeshSpec, eps: float = 0.0) -> np.ndarray:
    """Deconvolved, tapered long-range kernel at the offsets of the L = 2M
    box, [4][L][L][L] (components x, y, z, potential; residue order)."""
    M, h, s = spec.M, spec.h, spec.sigma
    Lb = 4 * M
    m = np.arange(Lb)
    m = np.where(m <= Lb // 2, m, m - Lb) * h
    Z, Y, X = np.meshgrid(m, m, m, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z + eps * eps)
    x = r / s
    with np.errstate(invalid="ignore", divide="ignore"):
        e_over_r = np.where(r > 0, erf(x) / np.where(r > 0, r, 1.0), 2.0 / (math.sqrt(math.pi) * s))
    chi = _taper(np.sqrt(X * X + Y * Y + Z * Z), math.sqrt(3.0) * M * h, 2 * M * h)
    pot = r * erf(x) + s / math.sqrt(math.pi) * np.exp(-x * x)
    f = np.fft.fftfreq(Lb)
    w1 = np.sinc(f) ** 8
    W2 = w1[:, None, None] * w1[None, :, None] * w1[None, None, :]
    L = 2 * M
    ml = np.arange(L)
    ml = np.where(ml < M, ml, ml - L) % Lb          # offsets -M < m < M (index M unused)
    out = np.zeros((4, L, L, L))
    for c, g in enumerate((X * e_over_r, Y * e_over_r, Z * e_over_r, pot)):
        gd = np.fft.irfftn(np.fft.rfftn(g * chi) / W2[:, :, :Lb // 2 + 1], s=(Lb, Lb, Lb),
                           axes=(0, 1, 2))
        out[c] = gd[np.ix_(ml, ml, ml)]
        out[c][M, :, :] = 0.0
        out[c][:, M, :] = 0.0
        out[c][:, :, M] = 0.0
    return out


def mesh_long(K, spec: MeshSpec, eps: float = 0.0, kernel=None):
    """(L [N, 3], eL [N]): the long-range repulsion sums and potential sums
    at the samples (the potential includes the self term)."""
    K = np.asarray(K, np.float64).reshape(-1, 3)
    M = spec.M
    L = 2 * M
    if kernel is None:
        kernel = kernel_offsets(spec, eps)
    Q = np.zeros((L, L, L))
    Q[:M, :M, :M] = charges(K, spec)
    Qh = np.fft.rfftn(Q)
    first, w = spread_weights(K, spec)
    out = np.zeros((K.shape[0], 4))
    for c in range(4):
        phi = np.fft.irfftn(np.fft.rfftn(kernel[c]) * Qh, s=(L, L, L), axes=(0, 1, 2))[:M, :M, :M]
        for a in range(4):
            for b in range(4):
                for cc in range(4):
                    out[:, c] += (w[:, 0, a] * w[:, 1, b] * w[:, 2, cc] *
                                  phi[first[:, 2] + cc, first[:, 1] + b, first[:, 0] + a])
    return out[:, :3], out[:, 3]


def self_potential(spec: MeshSpec, eps: float = 0.0) -> float:
    """g(0) of the potential kernel: eps erf(eps/sigma) + sigma/sqrt(pi) exp(-eps^2/sigma^2)."""
    s = spec.sigma
    return eps * math.erf(eps / s) + s / math.sqrt(math.pi) * math.exp(-(eps / s) ** 2)
