"""Hyperparameter fitting (Eq. 1 gradient ascent): on a small problem whose
targets come from a smooth field, Adam on the GPU's stochastic MLL and
gradient raises the EXACT marginal likelihood of the oracle's dense D-SKI
matrix, and the fitted length scale moves from its start toward the
field's scale."""
import math

import numpy as np
import pytest

from synth import workloads as W
from tests._gpu_helpers import need_gpu, torch

pytestmark = pytest.mark.gpu


def _dense_mll(p, theta):
    from oracle.dski import DSKI as ODSKI, Grid
    from oracle.mll import mll_dense
    d = len(p["m"])
    ell = [math.exp(v) for v in theta[:d]]
    sf = math.exp(theta[d])
    s2 = math.exp(2 * theta[d + 1])
    orc = ODSKI(p["X"], Grid(p["m"], p["lo"], p["hi"]), ell, sf, s2, s2)
    return mll_dense(orc, p["y"])


def test_fit_raises_the_exact_marginal_likelihood():
    need_gpu()
    from paper_1810_12283_gb300 import DSKI
    from paper_1810_12283_gb300.train import fit
    p = W.sine2d(n=300)   # sin 2 pi x1 cos 2 pi x2 with gradients, 32 x 32 grid
    X = torch.tensor(p["X"], device="cuda")
    y = torch.tensor(p["y"], device="cuda")
    theta0 = [math.log(0.4), math.log(0.4), math.log(0.7), 0.5 * math.log(1e-2)]
    op = DSKI(X, p["m"], p["lo"], p["hi"], [0.4, 0.4], 0.7, 1e-2, 1e-2)
    theta, hist = fit(op, y, theta0, steps=25, lr=0.08, rank=40, probes=16, seed=11)
    op.close()
    L0 = _dense_mll(p, theta0)
    L1 = _dense_mll(p, theta.tolist())
    assert L1 > L0 + 0.05 * abs(L0), (L0, L1)
    # the GPU's first value estimates the exact one (SLQ log det)
    assert abs(hist[0][0] - L0) <= 0.05 * abs(L0), (hist[0][0], L0)
    # the length scales shrink toward the field's (0.25 period scale)
    assert max(theta[0].item(), theta[1].item()) < math.log(0.4)
