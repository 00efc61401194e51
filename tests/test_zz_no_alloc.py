"""sparkling_grad_noalloc: the gradient computed in the library's fixed
scratch array, for callers that cannot let the library allocate device
memory (their memory belongs to their own pool or budget).  Its result must
match sparkling_grad's and the FP64 oracle's within the gradient tolerance of
the other tests, on consecutive calls that reuse the same scratch array.

This file is collected last on purpose: its first call sets the scratch
array up on the device, and it must pass both in a fresh process and after
every other test."""
import ctypes

import numpy as np
import pytest

import inputs
import oracle
from gpu_util import assert_grad_close

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


def call_noalloc(sp, K, grid, G, acc=0):
    """Direct C-ABI call of sparkling_grad_noalloc."""
    code = sp.lib().sparkling_grad_noalloc(
        ctypes.c_void_p(K.data_ptr()), sp._dtype_code(K), K.shape[0], ctypes.byref(grid), acc,
        ctypes.c_void_p(G.data_ptr()), sp._dtype_code(G),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return code


def case(seed, N, n, dtype):
    rng = np.random.default_rng(seed)
    K = rng.uniform(-0.5, 0.5, size=(N, 3)).astype(dtype)
    grid = inputs.density_gaussian(n, 0.2, 0.02)
    return K, grid


def test_noalloc_matches_grad_on_consecutive_calls(sp):
    """Three calls in a row on the shared scratch array: a large problem, then
    a smaller one with another grid and work split (which reads only what it
    has written, although the larger call left stale slots behind), then a
    large one again.  Each result matches sparkling_grad's and the oracle's
    (every target of the small problem, 512 random targets of the large
    ones), in FP64 and in FP32 output."""
    ctx = sp.sparkling_create(0)
    cases = ((2, 20000, 40, np.float32, 1, torch.float64),
             (1, 3000, 17, np.float64, 0, torch.float32),
             (3, 20000, 24, np.float32, 0, torch.float64))
    try:
        for seed, N, n, dt, acc, gdt in cases:
            K, g = case(seed, N, n, dt)
            Kd = torch.from_numpy(K).cuda()
            rho = torch.from_numpy(g.rho).cuda()
            grid = sp.make_grid(rho, g.lo, g.hi, g.n)
            G_ref = sp.sparkling_grad(ctx, Kd, grid, acc, G=torch.empty(N, 3, dtype=gdt,
                                                                           device="cuda"))
            sp.sparkling_status(ctx)
            G = torch.full((N, 3), float("nan"), dtype=gdt, device="cuda")
            assert call_noalloc(sp, Kd, grid, G, acc) == sp.OK, sp.sparkling_last_error(None)
            Gn = G.cpu().numpy().astype(np.float64)
            assert_grad_close(Gn, G_ref.cpu().numpy(), f"noalloc vs sparkling_grad (N = {N})")
            idx = (np.arange(N) if N <= 3000 else
                   np.sort(np.random.default_rng(seed).choice(N, size=512, replace=False)))
            _, _, G0 = oracle.forces(K.astype(np.float64), g, targets=idx)
            assert_grad_close(Gn[idx], G0, f"noalloc vs the oracle (N = {N})")
    finally:
        ctx.close()


def test_noalloc_rejects_problems_beyond_its_scratch(sp):
    K = torch.zeros(2_000_000, 3, dtype=torch.float32, device="cuda")
    rho = torch.ones(8, 8, 8, dtype=torch.float32, device="cuda")
    grid = sp.make_grid(rho)
    G = torch.empty_like(K)
    assert call_noalloc(sp, K, grid, G) == sp.E_INVAL
    msg = sp.sparkling_last_error(None)
    assert "scratch" in msg and "bytes" in msg
