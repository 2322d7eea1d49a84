"""Hyperparameter fitting by gradient ascent on the log marginal likelihood
(Eq. 1), as the paper's experiments fit the SE length scales, output scale
and noise before predicting.  Each step sets the hyperparameters, rebuilds
the pivoted-Cholesky preconditioner and evaluates L and dL/dtheta on the GPU
through the C ABI (MarginalLikelihood: PCG, SLQ and the grid adjoint); the
probes are fixed across steps (common random numbers), so the stochastic
objective is a deterministic function of theta.  Argument marshalling and
the optimiser's update only.
"""
import math

import torch

from .autograd import mll_function


def theta_of(op_hypers, d):
    """theta = (log l_1..d, log sigma_f, log sigma_n) from (ell list, sf, noise variance)."""
    ell, sf, nv = op_hypers
    return [math.log(v) for v in ell] + [math.log(sf), 0.5 * math.log(nv)]


def fit(op, y, theta0, steps=30, lr=0.05, rank=100, probes=16, seed=777, callback=None):
    """Adam ascent on L(theta).  Returns (theta, history of (L, theta)); the
    operator is left at the last evaluated hyperparameters."""
    theta = torch.tensor(list(theta0), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([theta], lr=lr)
    hist = []
    for it in range(steps):
        opt.zero_grad()
        L = mll_function(theta, op, y, rank=rank, probes=probes, seed=seed)
        (-L).backward()
        hist.append((float(L.detach()), theta.detach().clone()))
        if callback is not None:
            callback(it, float(L.detach()), theta.detach().clone())
        opt.step()
    return theta.detach(), hist
