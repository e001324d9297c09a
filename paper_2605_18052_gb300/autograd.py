"""torch.autograd.Function over the epipolar objective (the differentiation form of the path).

EpipolarLoss.apply(problem, R, c) evaluates the problem's objective (IRLS-weighted or L1,
Sec. "Epipolar Adjustment") at rotations R (N,3,3) and camera centres c (N,3), float64 CUDA
tensors. The forward call is one pass of the library's fused loss/adjoint kernels; the only
thing kept for backward is the per-camera gradient (N x 6), never a per-pair or per-point
quantity. With recompute=True the forward keeps nothing and backward runs the pass again.

Gradients: the library returns the left-trivialised gradient g_phi (R <- Exp(phi) R) and
g_c. For R the backward returns the tangent-space Euclidean gradient 0.5 [g_phi]_x R, whose
inner product with any rotation perturbation [dphi]_x R equals g_phi . dphi, so autograd
through any rotation parameterisation (exponential map, 6D, quaternions) is exact.
"""
from __future__ import annotations

import torch


def _hat(v: torch.Tensor) -> torch.Tensor:
    z = torch.zeros_like(v[:, 0])
    return torch.stack([torch.stack([z, -v[:, 2], v[:, 1]], -1),
                        torch.stack([v[:, 2], z, -v[:, 0]], -1),
                        torch.stack([-v[:, 1], v[:, 0], z], -1)], -2)


def _loss_grad(problem, R, c):
    R = R.detach().to(torch.float64).contiguous()
    c = c.detach().to(torch.float64).contiguous()
    problem.set_params_device(R, c)
    loss = torch.empty(1, dtype=torch.float64, device=R.device)
    grad = torch.empty(R.shape[0], 6, dtype=torch.float64, device=R.device)
    problem.loss_grad_device(loss, grad)
    return loss, grad


class EpipolarLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, problem, R, c, recompute: bool = False):
        loss, grad = _loss_grad(problem, R, c)
        ctx.problem = problem
        ctx.recompute = recompute
        if recompute:
            ctx.save_for_backward(R, c)
        else:
            ctx.save_for_backward(R, grad)
        return loss[0]

    @staticmethod
    def backward(ctx, grad_out):
        if ctx.recompute:
            R, c = ctx.saved_tensors
            _, grad = _loss_grad(ctx.problem, R, c)
        else:
            R, grad = ctx.saved_tensors
        g = grad * grad_out
        gR = 0.5 * _hat(g[:, :3]) @ R.to(torch.float64)
        return None, gR.to(R.dtype), g[:, 3:].to(R.dtype), None


def epipolar_loss(problem, R, c, recompute: bool = False) -> torch.Tensor:
    """Differentiable objective of `problem` (a binding.Problem) at (R, c)."""
    return EpipolarLoss.apply(problem, R, c, recompute)
