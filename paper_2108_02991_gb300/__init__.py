"""Python binding of libsparkling.so, the GB300 (sm_103a) library for the hot
path of full-3D SPARKLING (arxiv 2108.02991).

This module only marshals arguments: every function calls the C entry point
of the same name (declared in include/sparkling.h) with device pointers taken
from torch tensors and the current torch stream.  There is no fallback: if the
shared library is missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsparkling.so")

OK, E_INVAL, E_NOMEM, E_CUDA, E_NONFINITE, E_TIMEOUT, E_NOTCONV, E_IO, E_RANGE = range(9)
F32, F64 = 0, 1
ACC_KAHAN32, ACC_FP64, ACC_FP64_PAIR = 0, 1, 2
KERNEL_NAMES = ("pack", "attraction", "repulsion", "combine", "project", "engine", "driver", "step")
PROJECTION_FP64, PROJECTION_MIXED = 0, 1
BATCH_GRAPH = 1
BATCH_TWO_LAUNCHES = 2
STEP_AUTO, STEP_KERNELS, STEP_ENGINE = 0, 1, 2
STEP_PATHS = ("auto", "kernels", "engine")
ATTRACTION_DIRECT, ATTRACTION_FIELD = 0, 1
REPULSION_DIRECT, REPULSION_MESH = 0, 1

# Every entry point declared in include/sparkling.h.
ABI_SYMBOLS = (
    "sparkling_create", "sparkling_destroy", "sparkling_last_error", "sparkling_grad",
    "sparkling_energy", "sparkling_energy_backward", "sparkling_project", "sparkling_step",
    "sparkling_step_host", "sparkling_status", "sparkling_set_timing", "sparkling_kernel_times",
    "sparkling_launch_count", "sparkling_version", "sparkling_grad_noalloc",
    "sparkling_step_batched", "sparkling_set_autotune", "sparkling_tuning_report",
    "sparkling_set_attraction", "sparkling_attraction_field", "sparkling_set_regularisation",
    "sparkling_upsample", "sparkling_optimize", "sparkling_multires", "sparkling_set_repulsion",
    "sparkling_set_shape", "sparkling_set_projection", "sparkling_set_wait_budget",
    "sparkling_set_memory_limit", "sparkling_set_step_path",
)


class SparklingError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"[{code}] {message}")
        self.code = code


class Grid(ctypes.Structure):
    """sparkling_grid: rho device pointer, lo, hi, n = (nx, ny, nz)."""
    _fields_ = [("rho", ctypes.c_void_p), ("lo", ctypes.c_double), ("hi", ctypes.c_double),
                ("n", ctypes.c_int32 * 3), ("reserved", ctypes.c_int32)]


class Proj(ctypes.Structure):
    """sparkling_proj: constraint set and iteration control of the projection."""
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("box", ctypes.c_double),
                ("tol", ctypes.c_double), ("margin", ctypes.c_double),
                ("pin", ctypes.c_double * 3), ("pin_index", ctypes.c_int32),
                ("n_iter", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Mesh(ctypes.Structure):
    """sparkling_mesh: the fast repulsion's mesh."""
    _fields_ = [("lo", ctypes.c_double), ("hi", ctypes.c_double),
                ("sigma_cells", ctypes.c_double), ("rc_sigmas", ctypes.c_double),
                ("n_cells", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def make_mesh(n_cells, sigma_cells=2.5, rc_sigmas=4.0, lo=-0.5, hi=0.5) -> Mesh:
    m = Mesh()
    m.lo, m.hi = float(lo), float(hi)
    m.sigma_cells, m.rc_sigmas, m.n_cells = float(sigma_cells), float(rc_sigmas), int(n_cells)
    return m


class Schedule(ctypes.Structure):
    """sparkling_schedule: step schedule and level scaling of the driver."""
    _fields_ = [("eta", ctypes.c_double), ("eta_min", ctypes.c_double),
                ("eta_max", ctypes.c_double), ("alpha_factor", ctypes.c_double),
                ("beta_factor", ctypes.c_double), ("n_git", ctypes.c_int32),
                ("n_fixed", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


def make_schedule(eta, n_git, n_fixed=20, eta_min=1e-12, eta_max=1e3, alpha_factor=2.0,
                  beta_factor=4.0) -> Schedule:
    sc = Schedule()
    sc.eta, sc.eta_min, sc.eta_max = float(eta), float(eta_min), float(eta_max)
    sc.alpha_factor, sc.beta_factor = float(alpha_factor), float(beta_factor)
    sc.n_git, sc.n_fixed = int(n_git), int(n_fixed)
    return sc


_lib_handle = None


def lib() -> ctypes.CDLL:
    """Load libsparkling.so (raises if it has not been built)."""
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with paper_2108_02991_gb300.build.build() "
                "(or __graft_entry__.build()); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        p, i, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        sig = {
            "sparkling_create": ([ctypes.POINTER(p), i], i),
            "sparkling_destroy": ([p], None),
            "sparkling_last_error": ([p], ctypes.c_char_p),
            "sparkling_grad": ([p, p, i, i64, ctypes.POINTER(Grid), i, p, i, p, p, p], i),
            "sparkling_energy": ([p, p, i, i64, ctypes.POINTER(Grid), i, p, p, p, p], i),
            "sparkling_energy_backward": ([p, p, i, i64, ctypes.POINTER(Grid), i, p, d, p, i, p], i),
            "sparkling_project": ([p, p, i, i64, i64, ctypes.POINTER(Proj), p, p], i),
            "sparkling_step": ([p, p, i, i64, i64, ctypes.POINTER(Grid), i, d, ctypes.POINTER(Proj), p], i),
            "sparkling_step_host": ([p, p, i, i64, i64, ctypes.POINTER(Grid), p, i, d,
                                     ctypes.POINTER(Proj), p], i),
            "sparkling_status": ([p, p], i),
            "sparkling_set_timing": ([p, i], i),
            "sparkling_kernel_times": ([p, p, p, i, i], i),
            "sparkling_launch_count": ([p], i64),
            "sparkling_version": ([], ctypes.c_char_p),
            "sparkling_grad_noalloc": ([p, i, i64, ctypes.POINTER(Grid), i, p, i, p], i),
            "sparkling_set_autotune": ([p, i], i),
            "sparkling_set_shape": ([p, i, i], i),
            "sparkling_tuning_report": ([p, p, i64], i),
            "sparkling_set_attraction": ([p, i], i),
            "sparkling_attraction_field": ([p, p, p], i),
            "sparkling_set_regularisation": ([p, ctypes.c_double], i),
            "sparkling_set_projection": ([p, i], i),
            "sparkling_set_step_path": ([p, i], i),
            "sparkling_set_wait_budget": ([p, i64], i),
            "sparkling_set_memory_limit": ([p, i64], i),
            "sparkling_set_repulsion": ([p, i, p], i),
            "sparkling_upsample": ([p, p, p, i, i64, i64, p], i),
            "sparkling_optimize": ([p, p, i, i64, i64, p, p, i, p, p, p], i),
            "sparkling_multires": ([p, p, i, i64, i64, p, p, i, p, ctypes.c_int32, ctypes.c_char_p,
                                    p, p], i),
            "sparkling_step_batched": ([p, ctypes.c_int32, p, p, i, ctypes.c_int32,
                                        ctypes.POINTER(Grid), p, ctypes.POINTER(Proj), i, i, p], i),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib_handle = L
    return _lib_handle


def _check(ctx, code: int):
    if code != OK:
        msg = lib().sparkling_last_error(ctx.handle if ctx is not None else None)
        raise SparklingError(code, msg.decode() if msg else "unknown error")


class Context:
    """Owns a sparkling_ctx (device workspace, timing state)."""

    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        code = lib().sparkling_create(ctypes.byref(h), int(device))
        if code != OK:
            raise SparklingError(code, lib().sparkling_last_error(None).decode())
        self.handle = h
        self.device = int(device)

    def close(self):
        if getattr(self, "handle", None):
            lib().sparkling_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sparkling_create(device: int = 0) -> Context:
    return Context(device)


def sparkling_destroy(ctx: Context) -> None:
    ctx.close()


def sparkling_last_error(ctx: Optional[Context] = None) -> str:
    return lib().sparkling_last_error(ctx.handle if ctx else None).decode()


def sparkling_version() -> str:
    return lib().sparkling_version().decode()


# --- marshalling helpers ----------------------------------------------------

def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    raise TypeError(f"expected float32 or float64, got {t.dtype}")


def _dev_ptr(t, what: str):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def make_grid(rho, lo: float = -0.5, hi: float = 0.5, n: Optional[Sequence[int]] = None) -> Grid:
    """sparkling_grid for a float32 density tensor [nz, ny, nx] (device or,
    for the host entry points, any) -- n defaults to rho's shape."""
    if n is None:
        nz, ny, nx = rho.shape
        n = (nx, ny, nz)
    g = Grid()
    g.rho = ctypes.c_void_p(rho.data_ptr()) if (rho is not None and rho.is_cuda) else None
    g._rho_ref = rho        # the struct holds a raw pointer: keep the tensor alive with it
    g.lo, g.hi = float(lo), float(hi)
    for a in range(3):
        g.n[a] = int(n[a])
    return g


def make_proj(alpha, beta, box=0.5, n_iter=100, pin_index=-1, pin=(0.0, 0.0, 0.0), tol=0.0,
              margin=0.0, check_every=10) -> Proj:
    p = Proj()
    p.alpha, p.beta, p.box = float(alpha), float(beta), float(box)
    p.tol, p.margin = float(tol), float(margin)
    for c in range(3):
        p.pin[c] = float(pin[c])
    p.pin_index, p.n_iter, p.check_every = int(pin_index), int(n_iter), int(check_every)
    return p


def _rows(K) -> int:
    if K.dim() != 2 or K.shape[1] != 3:
        raise ValueError("K must have shape [N, 3]")
    return int(K.shape[0])


# --- entry points -------------------------------------------------------------

def sparkling_grad(ctx: Context, K, grid: Grid, acc: int = ACC_KAHAN32, G=None, A=None, R=None,
                   stream=None):
    """G = A - R for every sample (asynchronous); returns G."""
    import torch
    N = _rows(K)
    if G is None:
        G = torch.empty_like(K)
    _check(ctx, lib().sparkling_grad(ctx.handle, _dev_ptr(K, "K"), _dtype_code(K), N,
                                     ctypes.byref(grid), acc, _dev_ptr(G, "G"), _dtype_code(G),
                                     _dev_ptr(A, "A"), _dev_ptr(R, "R"), _stream(stream)))
    return G


def sparkling_grad_noalloc(K, grid: Grid, acc: int = ACC_KAHAN32, G=None, stream=None):
    """G = A - R using only the library's fixed 32 MiB scratch array (no
    device allocation by the library; blocks on the stream).  For callers
    whose device memory is owned by their own pool or budget."""
    import torch
    N = _rows(K)
    if G is None:
        G = torch.empty_like(K)
    _check(None, lib().sparkling_grad_noalloc(_dev_ptr(K, "K"), _dtype_code(K), N,
                                              ctypes.byref(grid), acc, _dev_ptr(G, "G"),
                                              _dtype_code(G), _stream(stream)))
    return G


def sparkling_energy(ctx: Context, K, grid: Grid, acc: int = ACC_KAHAN32, stream=None):
    """(F, F^a, F^r) as Python floats (blocks on the stream)."""
    F, Fa, Fr = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().sparkling_energy(ctx.handle, _dev_ptr(K, "K"), _dtype_code(K), _rows(K),
                                       ctypes.byref(grid), acc, ctypes.byref(F), ctypes.byref(Fa),
                                       ctypes.byref(Fr), _stream(stream)))
    return F.value, Fa.value, Fr.value


def sparkling_energy_backward(ctx: Context, K, grid: Grid, g=None, scale: float = 1.0,
                              acc: int = ACC_KAHAN32, dK=None, stream=None):
    """dK = scale * g * (A - R) / N with g a float64 device scalar tensor (or None)."""
    import torch
    if dK is None:
        dK = torch.empty_like(K)
    if g is not None and g.dtype != torch.float64:
        raise TypeError("g must be a float64 tensor")
    _check(ctx, lib().sparkling_energy_backward(
        ctx.handle, _dev_ptr(K, "K"), _dtype_code(K), _rows(K), ctypes.byref(grid), acc,
        _dev_ptr(g, "g"), float(scale), _dev_ptr(dK, "dK"), _dtype_code(dK), _stream(stream)))
    return dK


def sparkling_project(ctx: Context, K, Nc: int, Ns: int, proj: Proj, want_violation: bool = False,
                      stream=None):
    """Project every shot of K in place; returns the (amplitude, slew, box,
    pin) violations of the result when asked (blocks then)."""
    v = (ctypes.c_double * 4)() if want_violation else None
    _check(ctx, lib().sparkling_project(ctx.handle, _dev_ptr(K, "K"), _dtype_code(K), int(Nc),
                                        int(Ns), ctypes.byref(proj), v, _stream(stream)))
    return list(v) if want_violation else None


def sparkling_step(ctx: Context, K, Nc: int, Ns: int, grid: Grid, eta: float, proj: Proj,
                   acc: int = ACC_KAHAN32, stream=None):
    """K <- Pi(K - eta G) in place (asynchronous unless converged mode)."""
    _check(ctx, lib().sparkling_step(ctx.handle, _dev_ptr(K, "K"), _dtype_code(K), int(Nc),
                                     int(Ns), ctypes.byref(grid), acc, float(eta),
                                     ctypes.byref(proj), _stream(stream)))


def sparkling_step_batched(ctx: Context, K, traj_off: Sequence[int], Ns: int,
                           grids: Sequence[Grid], etas: Sequence[float], projs: Sequence[Proj],
                           acc: int = ACC_KAHAN32, graph: bool = True, one_launch: bool = True,
                           stream=None):
    """One projected-gradient step of B trajectories (samples
    [traj_off[b], traj_off[b+1]) of K), in place, in one persistent launch;
    one_launch=False runs the symmetric repulsion in its own kernel first."""
    B = len(grids)
    if len(traj_off) != B + 1 or len(etas) != B or len(projs) != B:
        raise ValueError("traj_off needs B+1 entries, etas and projs B")
    off = (ctypes.c_int64 * (B + 1))(*[int(v) for v in traj_off])
    garr = (Grid * B)(*grids)
    earr = (ctypes.c_double * B)(*[float(v) for v in etas])
    parr = (Proj * B)(*projs)
    _check(ctx, lib().sparkling_step_batched(ctx.handle, B, off, _dev_ptr(K, "K"), _dtype_code(K),
                                             int(Ns), garr, earr, parr, acc,
                                             (BATCH_GRAPH if graph else 0) |
                                             (0 if one_launch else BATCH_TWO_LAUNCHES),
                                             _stream(stream)))


def sparkling_step_host(ctx: Context, K_host, Nc: int, Ns: int, grid: Grid, rho_host, eta: float,
                        proj: Proj, acc: int = ACC_KAHAN32, stream=None):
    """sparkling_step on host tensors (CPU, contiguous; pinned for async DMA)."""
    for t, what in ((K_host, "K_host"), (rho_host, "rho_host")):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{what} must be a contiguous host tensor")
    _check(ctx, lib().sparkling_step_host(ctx.handle, ctypes.c_void_p(K_host.data_ptr()),
                                          _dtype_code(K_host), int(Nc), int(Ns), ctypes.byref(grid),
                                          ctypes.c_void_p(rho_host.data_ptr()), acc, float(eta),
                                          ctypes.byref(proj), _stream(stream)))


def sparkling_status(ctx: Context, stream=None) -> int:
    """Synchronise and raise if the device recorded an error since the last check."""
    code = lib().sparkling_status(ctx.handle, _stream(stream))
    _check(ctx, code)
    return code


def sparkling_set_timing(ctx: Context, enable: bool = True) -> None:
    _check(ctx, lib().sparkling_set_timing(ctx.handle, 1 if enable else 0))


def sparkling_kernel_times(ctx: Context, reset: bool = False):
    """{kernel kind: (total ms, launches)} since the last reset."""
    n = len(KERNEL_NAMES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    _check(ctx, lib().sparkling_kernel_times(ctx.handle, ms, cnt, n, 1 if reset else 0))
    return {KERNEL_NAMES[k]: (ms[k], cnt[k]) for k in range(n)}


def sparkling_set_autotune(ctx: Context, enable: int = 1) -> None:
    """1: tune tile shapes at first use (default); 0: default shapes; -1: retune."""
    _check(ctx, lib().sparkling_set_autotune(ctx.handle, int(enable)))


def sparkling_set_shape(ctx: Context, kernel: str, variant: int) -> None:
    """Pin the tile shape of "attraction" (0/1/2: 128/256/512 threads) or of
    the symmetric "repulsion" (0: 256 threads, 2 sources per lane, targets
    paired; 1: 256 threads, 4 sources, targets paired; 2: 256 threads, 2
    sources, sources paired; 3: 128 threads, 8 targets per lane, 2 sources,
    sources paired); -1 unpins."""
    _check(ctx, lib().sparkling_set_shape(ctx.handle, KERNEL_NAMES.index(kernel), int(variant)))


def sparkling_tuning_report(ctx: Context) -> str:
    buf = ctypes.create_string_buffer(8192)
    _check(ctx, lib().sparkling_tuning_report(ctx.handle, buf, len(buf)))
    return buf.value.decode()


def sparkling_set_attraction(ctx: Context, mode: int) -> None:
    """ATTRACTION_DIRECT (direct sum, default) or ATTRACTION_FIELD
    (interpolated node field of the density)."""
    _check(ctx, lib().sparkling_set_attraction(ctx.handle, int(mode)))


def sparkling_set_projection(ctx: Context, mode: int) -> None:
    """PROJECTION_FP64 (default: FP64 iteration for every K dtype) or
    PROJECTION_MIXED (FP32 K: FP32 iteration on the displacement)."""
    _check(ctx, lib().sparkling_set_projection(ctx.handle, int(mode)))


def sparkling_set_step_path(ctx: Context, path: str) -> None:
    """Device path of sparkling_step / sparkling_step_host: "auto" (the
    persistent engine from 2^22 samples on), "kernels" or "engine"."""
    _check(ctx, lib().sparkling_set_step_path(ctx.handle, STEP_PATHS.index(path)))


def sparkling_set_wait_budget(ctx: Context, cycles: int) -> None:
    """Budget of the context's bounded device waits in SM clock cycles
    (negative: the default, about 2 s)."""
    _check(ctx, lib().sparkling_set_wait_budget(ctx.handle, int(cycles)))


def sparkling_set_memory_limit(ctx: Context, nbytes: int) -> None:
    """Cap on the context's own device allocations (0: none)."""
    _check(ctx, lib().sparkling_set_memory_limit(ctx.handle, int(nbytes)))


def sparkling_set_regularisation(ctx: Context, eps: float) -> None:
    """Kernel H(r) = sqrt(r^2 + eps^2) for the context's later calls (0: |r|)."""
    _check(ctx, lib().sparkling_set_regularisation(ctx.handle, float(eps)))


def sparkling_set_repulsion(ctx: Context, mode: int, mesh: Optional[Mesh] = None) -> None:
    """REPULSION_DIRECT (every pair, default) or REPULSION_MESH (particle-
    particle particle-mesh summation on `mesh`)."""
    _check(ctx, lib().sparkling_set_repulsion(ctx.handle, int(mode),
                                              ctypes.byref(mesh) if mesh is not None else None))


def sparkling_attraction_field(ctx: Context, grid: Grid, stream=None) -> None:
    """(Re)build the node field of grid's density (blocking)."""
    _check(ctx, lib().sparkling_attraction_field(ctx.handle, ctypes.byref(grid),
                                                 _stream(stream)))


def sparkling_upsample(ctx: Context, Kc, Nc: int, d: int, Kf=None, stream=None):
    """L_{2d} between levels: [Nc*d, 3] -> [Nc*2d, 3] (a new tensor unless Kf)."""
    import torch
    if Kf is None:
        Kf = torch.empty(Nc * 2 * d, 3, dtype=Kc.dtype, device=Kc.device)
    _check(ctx, lib().sparkling_upsample(ctx.handle, _dev_ptr(Kc, "Kc"), _dev_ptr(Kf, "Kf"),
                                         _dtype_code(Kc), int(Nc), int(d), _stream(stream)))
    return Kf


def sparkling_optimize(ctx: Context, K, Nc: int, Ns: int, grid: Grid, proj: Proj,
                       sched: Schedule, acc: int = ACC_KAHAN32, stream=None):
    """n_git projected-gradient iterations (fixed step, then Barzilai-Borwein)
    on K in place; returns the list of steps."""
    trace = (ctypes.c_double * max(sched.n_git, 1))()
    _check(ctx, lib().sparkling_optimize(ctx.handle, _dev_ptr(K, "K"), _dtype_code(K), int(Nc),
                                         int(Ns), ctypes.byref(grid), ctypes.byref(proj), acc,
                                         ctypes.byref(sched), trace, _stream(stream)))
    return list(trace)[:sched.n_git]


def sparkling_multires(ctx: Context, K, Nc: int, Ns: int, grid: Grid, proj: Proj,
                       sched: Schedule, start_level: int, acc: int = ACC_KAHAN32,
                       checkpoint_prefix: Optional[str] = None, stream=None):
    """Algorithm 1 from level start_level to the full resolution.  K is a
    buffer of Nc*Ns rows whose first Nc*(Ns >> start_level) rows hold the
    initial pattern; returns the steps [levels][n_git]."""
    levels = start_level + 1
    trace = (ctypes.c_double * max(levels * sched.n_git, 1))()
    pre = checkpoint_prefix.encode() if checkpoint_prefix else None
    _check(ctx, lib().sparkling_multires(ctx.handle, _dev_ptr(K, "K"), _dtype_code(K), int(Nc),
                                         int(Ns), ctypes.byref(grid), ctypes.byref(proj), acc,
                                         ctypes.byref(sched), int(start_level), pre, trace,
                                         _stream(stream)))
    n = sched.n_git
    return [list(trace)[l * n:(l + 1) * n] for l in range(levels)]


def read_checkpoint(path: str):
    """(level, Nc, samples per shot, numpy array [Nc*Ns_l, 3]) of a checkpoint file."""
    import numpy as np
    with open(path, "rb") as f:
        head = f.read(64)
        if head[:8] != b"SPKLCKPT":
            raise ValueError(f"{path} is not a checkpoint")
        version, nc, ns, level, dtype = np.frombuffer(head[8:48], dtype=np.int64)
        if version != 1:
            raise ValueError(f"unknown checkpoint version {version}")
        arr = np.frombuffer(f.read(), dtype=np.float32 if dtype == F32 else np.float64)
    return int(level), int(nc), int(ns), arr.reshape(-1, 3).copy()


def sparkling_launch_count(ctx: Context) -> int:
    return int(lib().sparkling_launch_count(ctx.handle))


from .autograd import SparklingEnergy, sparkling_energy_fn  # noqa: E402,F401
