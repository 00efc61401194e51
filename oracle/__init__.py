"""FP64 CPU oracle for the SPARKLING hot path (arxiv 2108.02991).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It never imports the
CUDA library and the CUDA library never imports it; the two share no code.

The arithmetic lives in ``sparkling_oracle.c`` (plain C, IEEE double,
``-ffp-contract=off``); this module only builds it with gcc and marshals
NumPy arrays.  See the C file for the definitions followed:

* ``forces``  -- A_i, R_i, G_i = A_i - R_i (Sec. II-C, eqs. attraction_term,
  repulsion_term, attraction_derivative_basic, Fr_grad with H = |.|_2);
* ``energy``  -- F^a, F^r (eqs. global_minimization, attraction_term,
  repulsion_term);
* ``energy_terms`` -- the terms of F that contain one sample, with that
  sample moved (for central differences of F in one coordinate);
* ``attraction_at`` -- attraction force and potential of the density at
  arbitrary points (the field of eq. attraction_derivative_basic);
* ``project`` -- per-shot projection onto the constraint set (eq. constraints,
  Sec. II-D, Suppl. Sec. I) by FISTA on the dual;
* ``violation`` -- the constraint checker;
* ``step``    -- one projected-gradient step (eq. proj_grad_descent).

Fast repulsion (the exact particle-mesh split of the kernel):

* ``repulsion_split`` -- exact short-range (erfc, cut at rc) and long-range
  (erf) parts of the repulsion and of its distance sums.

Algorithm 1 (multi-resolution SPARKLING):

* ``upsample`` -- the linear interpolator L_{2d} between levels;
* ``optimize`` -- n_git projected-gradient iterations at one resolution,
  fixed step then Barzilai-Borwein (Sec. II-C, choice of step size);
* ``multires`` -- the level loop with per-level constraint scaling.

``forces``, ``energy``, ``attraction_at`` and ``step`` take ``eps`` for the
regularised kernel H(r) = sqrt(r^2 + eps^2) (Sec. II-C, choice of step size).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sparkling_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOTCONV = 0, 1, 6


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP, -O2, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            d, i64, p = ctypes.c_double, ctypes.c_int64, ctypes.c_void_p
            lib.oracle_forces.argtypes = [p, i64, p, i64, i64, i64, d, d, p, i64, p, p, p, p, p, d]
            lib.oracle_energy.argtypes = [p, i64, p, i64, i64, i64, d, d, p, p, d]
            lib.oracle_energy_terms.argtypes = [p, i64, p, i64, i64, i64, d, d, p, p, i64, p, p, d]
            lib.oracle_energy_terms.restype = ctypes.c_int
            lib.oracle_project.argtypes = [p, p, i64, i64, d, d, d, i64, p, i64, d, d, i64, p]
            lib.oracle_violation.argtypes = [p, i64, i64, d, d, d, i64, p, p]
            lib.oracle_step.argtypes = [p, i64, i64, p, i64, i64, i64, d, d, d, d, d, d, i64, p, i64, d]
            lib.oracle_attraction_at.argtypes = [p, i64, p, i64, i64, i64, d, d, p, p, d]
            lib.oracle_attraction_at.restype = ctypes.c_int
            lib.oracle_upsample.argtypes = [p, i64, i64, p]
            lib.oracle_optimize.argtypes = [p, i64, i64, p, i64, i64, i64, d, d, d, d, d, i64, p,
                                            i64, i64, i64, d, d, d, d, p]
            lib.oracle_multires.argtypes = [p, i64, i64, p, i64, i64, i64, d, d, d, d, d, i64, p,
                                            i64, i64, i64, i64, d, d, d, d, d, d, p, p]
            lib.oracle_repulsion_split.argtypes = [p, i64, d, d, d, p, i64, p, p, p, p]
            for f in (lib.oracle_upsample, lib.oracle_optimize, lib.oracle_multires,
                      lib.oracle_repulsion_split):
                f.restype = ctypes.c_int
            for f in (lib.oracle_forces, lib.oracle_energy, lib.oracle_project,
                      lib.oracle_violation, lib.oracle_step):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _grid_args(grid):
    rho = _f64(grid.rho)
    nx, ny, nz = (int(v) for v in grid.n)
    if rho.size != nx * ny * nz:
        raise ValueError("rho size does not match grid.n")
    return rho, nx, ny, nz, float(grid.lo), float(grid.hi)


def forces(K, grid, targets=None, energies: bool = False, eps: float = 0.0):
    """Return (A, R, G) as float64 [M, 3] for the target indices (all if None);
    with ``energies`` also the per-target sums (ea, er).  eps > 0: kernel
    sqrt(r^2 + eps^2)."""
    K = _f64(K)
    N = K.shape[0]
    rho, nx, ny, nz, lo, hi = _grid_args(grid)
    if targets is None:
        tptr, M = None, N
    else:
        targets = np.ascontiguousarray(np.asarray(targets, dtype=np.int64))
        tptr, M = _ptr(targets), targets.size
    A = np.empty((M, 3)); R = np.empty((M, 3)); G = np.empty((M, 3))
    ea = np.empty(M); er = np.empty(M)
    st = _load().oracle_forces(_ptr(K), N, _ptr(rho), nx, ny, nz, lo, hi, tptr, M,
                               _ptr(A), _ptr(R), _ptr(G), _ptr(ea), _ptr(er), float(eps))
    if st != OK:
        raise ValueError(f"oracle_forces failed ({st})")
    return (A, R, G, ea, er) if energies else (A, R, G)


def energy_terms(K, grid, idx, points, eps: float = 0.0):
    """(ea, er) for M pairs (idx[m], points[m]): the energy sums of sample
    idx[m] moved to points[m] -- sum_q rho_q |p - x_q| and sum_{j != i}
    |p - K_j|.  F depends on K_i only through ea / N - er / N^2."""
    K = _f64(K)
    rho, nx, ny, nz, lo, hi = _grid_args(grid)
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64).ravel())
    P = _f64(points).reshape(-1, 3)
    if P.shape[0] != idx.size:
        raise ValueError("one point per index")
    ea = np.empty(idx.size)
    er = np.empty(idx.size)
    st = _load().oracle_energy_terms(_ptr(K), K.shape[0], _ptr(rho), nx, ny, nz, lo, hi,
                                     _ptr(idx), _ptr(P), idx.size, _ptr(ea), _ptr(er), float(eps))
    if st != OK:
        raise ValueError(f"oracle_energy_terms failed ({st})")
    return ea, er


def attraction_at(points, grid, eps: float = 0.0):
    """(A, phi): attraction force [M, 3] and potential [M] of the density at
    arbitrary points (float64)."""
    P = _f64(points).reshape(-1, 3)
    rho, nx, ny, nz, lo, hi = _grid_args(grid)
    A = np.empty_like(P)
    phi = np.empty(P.shape[0])
    st = _load().oracle_attraction_at(_ptr(P), P.shape[0], _ptr(rho), nx, ny, nz, lo, hi,
                                      _ptr(A), _ptr(phi), float(eps))
    if st != OK:
        raise ValueError(f"oracle_attraction_at failed ({st})")
    return A, phi


def energy(K, grid, eps: float = 0.0):
    """Return (F, F^a, F^r)."""
    K = _f64(K)
    rho, nx, ny, nz, lo, hi = _grid_args(grid)
    fa, fr = ctypes.c_double(), ctypes.c_double()
    st = _load().oracle_energy(_ptr(K), K.shape[0], _ptr(rho), nx, ny, nz, lo, hi,
                               ctypes.byref(fa), ctypes.byref(fr), float(eps))
    if st != OK:
        raise ValueError(f"oracle_energy failed ({st})")
    return fa.value - fr.value, fa.value, fr.value


def project(K, Nc, Ns, alpha, beta, box=0.5, pin_index=-1, pin=(0.0, 0.0, 0.0), n_iter=100,
            tol=0.0, margin=0.0, check_every=10, return_iters=False):
    """Project each of Nc shots of Ns samples; returns a new float64 [N, 3]
    (and the per-shot iteration counts).  Raises on invalid input; in
    converged mode (tol > 0) a shot that did not converge raises RuntimeError."""
    K = _f64(K).reshape(-1, 3)
    if K.shape[0] != Nc * Ns:
        raise ValueError("K must hold Nc*Ns samples")
    out = np.empty_like(K)
    pin_a = _f64(pin)
    iters = np.zeros(max(Nc, 1), dtype=np.int64)
    st = _load().oracle_project(_ptr(K), _ptr(out), Nc, Ns, alpha, beta, box, pin_index,
                                _ptr(pin_a), n_iter, tol, margin, check_every, _ptr(iters))
    if st == ENOTCONV:
        raise RuntimeError("oracle projection did not converge")
    if st != OK:
        raise ValueError(f"oracle_project failed ({st})")
    return (out, iters[:Nc]) if return_iters else out


def violation(K, Nc, Ns, alpha, beta, box=0.5, pin_index=-1, pin=(0.0, 0.0, 0.0)):
    """Largest (amplitude, slew, box, pin) violation over all shots."""
    K = _f64(K).reshape(-1, 3)
    out = np.zeros(4)
    pin_a = _f64(pin)
    st = _load().oracle_violation(_ptr(K), Nc, Ns, alpha, beta, box, pin_index, _ptr(pin_a),
                                  _ptr(out))
    if st != OK:
        raise ValueError(f"oracle_violation failed ({st})")
    return out


def step(K, Nc, Ns, grid, eta, alpha, beta, box=0.5, pin_index=-1, pin=(0.0, 0.0, 0.0),
         n_iter=100, eps: float = 0.0):
    """One projected-gradient step K <- Pi(K - eta G); returns a new array."""
    K = _f64(K).reshape(-1, 3).copy()
    rho, nx, ny, nz, lo, hi = _grid_args(grid)
    pin_a = _f64(pin)
    st = _load().oracle_step(_ptr(K), Nc, Ns, _ptr(rho), nx, ny, nz, lo, hi, eta, alpha, beta,
                             box, pin_index, _ptr(pin_a), n_iter, float(eps))
    if st != OK:
        raise ValueError(f"oracle_step failed ({st})")
    return K


def upsample(K, Nc, d):
    """L_{2d}: [Nc*d, 3] -> [Nc*2d, 3] (float64)."""
    Kc = _f64(K).reshape(-1, 3)
    if Kc.shape[0] != Nc * d:
        raise ValueError("K must hold Nc*d samples")
    out = np.empty((Nc * 2 * d, 3))
    if _load().oracle_upsample(_ptr(Kc), Nc, d, _ptr(out)) != OK:
        raise ValueError("oracle_upsample failed")
    return out


def optimize(K, Nc, Ns, grid, alpha, beta, box=0.5, pin_index=-1, pin=(0.0, 0.0, 0.0),
             n_pit=100, n_git=10, n_fixed=20, eta=1e-3, eta_min=1e-12, eta_max=1e3, eps=0.0):
    """n_git projected-gradient iterations at one resolution; returns
    (K float64 [Nc*Ns, 3], steps [n_git])."""
    Kw = _f64(K).reshape(-1, 3).copy()
    if Kw.shape[0] != Nc * Ns:
        raise ValueError("K must hold Nc*Ns samples")
    rho, nx, ny, nz, lo, hi = _grid_args(grid)
    pin_a = _f64(pin)
    trace = np.zeros(max(n_git, 1))
    st = _load().oracle_optimize(_ptr(Kw), Nc, Ns, _ptr(rho), nx, ny, nz, lo, hi, alpha, beta, box,
                                 pin_index, _ptr(pin_a), n_pit, n_git, n_fixed, eta, eta_min,
                                 eta_max, eps, _ptr(trace))
    if st != OK:
        raise ValueError(f"oracle_optimize failed ({st})")
    return Kw, trace[:n_git]


def multires(K, Nc, Ns, grid, alpha, beta, box=0.5, pin_index=-1, pin=(0.0, 0.0, 0.0), n_pit=100,
             start_level=0, n_git=10, n_fixed=20, eta=1e-3, eta_min=1e-12, eta_max=1e3,
             alpha_factor=2.0, beta_factor=4.0, eps=0.0):
    """Algorithm 1 from level start_level (K holds Nc * (Ns >> start_level)
    samples) to the full resolution; returns (K [Nc*Ns, 3], [K of every
    level before up-sampling], steps [levels, n_git])."""
    Kc = _f64(K).reshape(-1, 3)
    if Kc.shape[0] != Nc * (Ns >> start_level):
        raise ValueError("K must hold Nc * (Ns >> start_level) samples")
    Kw = np.zeros((Nc * Ns, 3))
    Kw[:Kc.shape[0]] = Kc
    levels = list(range(start_level, -1, -1))
    sizes = [Nc * (Ns >> l) for l in levels]
    lev = np.zeros((sum(sizes), 3))
    trace = np.zeros((len(levels), max(n_git, 1)))
    rho, nx, ny, nz, lo, hi = _grid_args(grid)
    pin_a = _f64(pin)
    st = _load().oracle_multires(_ptr(Kw), Nc, Ns, _ptr(rho), nx, ny, nz, lo, hi, alpha, beta, box,
                                 pin_index, _ptr(pin_a), n_pit, start_level, n_git, n_fixed, eta,
                                 eta_min, eta_max, alpha_factor, beta_factor, eps, _ptr(lev),
                                 _ptr(trace))
    if st != OK:
        raise ValueError(f"oracle_multires failed ({st})")
    out, o = [], 0
    for n in sizes:
        out.append(lev[o:o + n].copy())
        o += n
    return Kw, out, trace[:, :n_git]


def repulsion_split(K, sigma, rc=0.0, eps=0.0, targets=None):
    """(S, L, eS, eL): exact short-range (pairs closer than rc; rc <= 0: all)
    and long-range parts of the repulsion sums and distance sums (not
    scaled by 1/N) for the target indices (all if None)."""
    K = _f64(K).reshape(-1, 3)
    N = K.shape[0]
    if targets is None:
        tptr, M = None, N
    else:
        targets = np.ascontiguousarray(np.asarray(targets, dtype=np.int64))
        tptr, M = _ptr(targets), targets.size
    S = np.empty((M, 3)); L = np.empty((M, 3)); eS = np.empty(M); eL = np.empty(M)
    st = _load().oracle_repulsion_split(_ptr(K), N, float(sigma), float(rc), float(eps), tptr, M,
                                        _ptr(S), _ptr(L), _ptr(eS), _ptr(eL))
    if st != OK:
        raise ValueError(f"oracle_repulsion_split failed ({st})")
    return S, L, eS, eL
