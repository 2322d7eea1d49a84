"""torch.autograd.Function for the log marginal likelihood of Eq. 1.

Forward evaluates L(theta) = -1/2 [y^T K~^-1 y + log|K~| + N log 2 pi] for
theta = (log l_1, ..., log l_d, log sigma_f, log sigma_n) through the C ABI
(dski_set_hypers, pivchol_build, dski_mll_grad: PCG solves, stochastic
Lanczos log determinant and the grid adjoint of the Kronecker products all
run on the GPU); backward returns grad_out * dL/dtheta from the same call.
Argument marshalling only -- no arithmetic of the method happens here.
"""
import math

import torch

from . import _lib


class MarginalLikelihood(torch.autograd.Function):
    """L(theta) for a fixed D-SKI operator `op` (its points and grid) and targets y.

    theta: float64 tensor of d + 2 entries (log length scales, log output
    scale, log noise standard deviation; the gradient-row noise keeps the
    operator's ratio to the value-row noise)."""

    @staticmethod
    def forward(ctx, theta, op, y, rank, probes, seed, rtol=None, maxit=100000):
        th = [float(v) for v in theta.detach().cpu().tolist()]
        d = op.d
        if len(th) != d + 2:
            raise ValueError(f"theta needs {d + 2} entries, got {len(th)}")
        ell = [math.exp(v) for v in th[:d]]
        sf = math.exp(th[d])
        s2 = math.exp(2.0 * th[d + 1])
        op.set_hypers(ell, sf, s2, s2 * op.noise_ratio)
        pc = op.pivchol(rank)
        try:
            mll, grad = op.mll_grad(y, pc, probes=probes, seed=seed, rtol=rtol, maxit=maxit)
        finally:
            pc.close()
        ctx.save_for_backward(torch.tensor(grad, dtype=theta.dtype, device=theta.device))
        return torch.tensor(mll, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None, None, None, None, None


def mll_function(theta, op, y, rank=100, probes=16, seed=777, rtol=None, maxit=100000):
    """Differentiable log marginal likelihood (Eq. 1) of the D-SKI model.
    rtol / maxit: the batched PCG's stopping rule (default: dski_mll_grad's
    1e-8 and 100,000 iterations)."""
    _lib.load()
    return MarginalLikelihood.apply(theta, op, y, rank, probes, seed, rtol, maxit)
