"""The attraction-repulsion energy as a torch.autograd.Function.

forward  = sparkling_energy: F = F^a - F^r (paper eqs. global_minimization,
           attraction_term, repulsion_term), a float64 scalar on K's device;
backward = sparkling_energy_backward: dL/dK = dL/dF * (A - R) / N
           (eqs. attraction_derivative_basic and Fr_grad), computed by the
           gradient kernel with the per-pair distances recomputed -- nothing
           of size N x N (or N x P) is ever stored; only K and the density
           grid are kept for the backward.
"""
from __future__ import annotations

import torch


class SparklingEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx_, K, rho, lo, hi, lib_ctx, acc):
        from . import make_grid, sparkling_energy
        grid = make_grid(rho, lo, hi)
        F, _, _ = sparkling_energy(lib_ctx, K, grid, acc)
        ctx_.save_for_backward(K, rho)
        ctx_.lo, ctx_.hi, ctx_.lib_ctx, ctx_.acc = lo, hi, lib_ctx, acc
        return torch.tensor(F, dtype=torch.float64, device=K.device)

    @staticmethod
    def backward(ctx_, grad_out):
        from . import make_grid, sparkling_energy_backward
        K, rho = ctx_.saved_tensors
        grid = make_grid(rho, ctx_.lo, ctx_.hi)
        g = grad_out.detach().to(torch.float64).contiguous()
        dK = sparkling_energy_backward(ctx_.lib_ctx, K, grid, g=g, scale=1.0, acc=ctx_.acc)
        return dK, None, None, None, None, None


def sparkling_energy_fn(K, rho, lib_ctx, lo: float = -0.5, hi: float = 0.5, acc: int = 0):
    """F(K) differentiable with respect to K (CUDA tensor [N, 3])."""
    return SparklingEnergy.apply(K, rho, lo, hi, lib_ctx, acc)
