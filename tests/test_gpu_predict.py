"""GPU parity of prediction (Sec. 5; the D-SKI cross-covariance of Sec. 3.1)
against the FP64 oracle (oracle/predict.py).

* mean and gradient at test points, mu* = [W*; dW*] K_UU [W; dW]^T alpha, for
  the same alpha, within the normwise bound of the product evaluated term by
  term: 64 u || |B*| K_UU |B|^T |alpha| || / ||mu*|| (Higham, Sec. 3.5;
  u = 2^-53 on every path: prediction runs in FP64 arithmetic in every mode,
  and FP64_TC's digit products are held to the FP64 bar).  alpha = K~^-1 y
  of an ill-conditioned system carries entries far above mu*, so this
  condition number, not 1, sets the scale.  Every element is also held to
  the componentwise bound gamma_K (|B*| K_UU |B|^T |alpha|)_i;
* the preconditioner variance estimate s_f^2 - k_x^T M^-1 k_x with the
  GPU's own pivots rebuilt in the oracle: 1e-9 relative;
* d = 2 and d = 3, grid-form (d = 2, M < N) and Q1-form preconditioners, and
  test points without a full stencil (DSKI_ERR_OUT_OF_GRID).
"""
import numpy as np
import pytest

from synth import workloads as W
from tests._gpu_helpers import (gpu_op, oracle_op, need_gpu, rel, torch, elem_err,
                                elem_tolerance)

pytestmark = pytest.mark.gpu


def _test_points(p, k, seed):
    rng = np.random.default_rng(seed)
    lo = np.asarray(p["X"]).min(axis=0)
    hi = np.asarray(p["X"]).max(axis=0)
    return rng.uniform(lo, hi, (k, len(p["m"])))


def _abs_mean(orc, alpha, Xs):
    """|B*| K_UU |B|^T |alpha|: the mean's terms in absolute value."""
    from oracle.dski import interp_matrix, kuu_apply
    Bs = abs(interp_matrix(Xs, orc.grid))
    return Bs @ kuu_apply(orc.grid, orc.ell, orc.sf, (abs(orc.B).T @ np.abs(alpha))[:, None])[:, 0]


def _mean_tolerance(orc, alpha, Xs, u):
    from oracle.predict import dski_mean
    a = _abs_mean(orc, alpha, Xs)
    ref = dski_mean(orc, alpha, Xs)
    return max(1e-13, 64 * u * np.linalg.norm(a) / np.linalg.norm(ref))


@pytest.mark.parametrize("make,prec", [
    (lambda: W.sine2d(), "fp64"),
    (lambda: W.sine2d(), "fp64_tc"),
    (lambda: W.sine2d(), "mixed_3xtf32"),
    (lambda: W.small3d(40, m=9, seed=3), "fp64"),
], ids=["sine2d-fp64", "sine2d-fp64_tc", "sine2d-mixed", "3d-fp64"])
def test_predictive_mean_and_gradient(make, prec):
    need_gpu()
    from oracle.predict import dski_mean
    p = make()
    orc = oracle_op(p)
    alpha = np.linalg.solve(orc.dense(), p["y"])
    Xs = _test_points(p, 37, 11)
    want = dski_mean(orc, alpha, Xs)
    tol = _mean_tolerance(orc, alpha, Xs, 2.0**-53)
    etol = elem_tolerance(orc, "fp64")
    op = gpu_op(p, prec)
    mean, var = op.predict(torch.tensor(alpha, device="cuda"), torch.tensor(Xs, device="cuda"))
    assert var is None
    assert rel(mean.cpu().numpy(), want) <= tol, (rel(mean.cpu().numpy(), want), tol)
    ee = elem_err(mean.cpu().numpy(), want, _abs_mean(orc, alpha, Xs))
    assert ee <= etol, (ee, etol)
    # a well-conditioned alpha (random): the same bound is tight here
    a2 = np.random.default_rng(5).normal(size=orc.N)
    tol2 = _mean_tolerance(orc, a2, Xs, 2.0**-53)
    m2, _ = op.predict(torch.tensor(a2, device="cuda"), torch.tensor(Xs, device="cuda"))
    got2 = rel(m2.cpu().numpy(), dski_mean(orc, a2, Xs))
    assert got2 <= tol2 and tol2 < 1e-9, (got2, tol2)
    assert elem_err(m2.cpu().numpy(), dski_mean(orc, a2, Xs), _abs_mean(orc, a2, Xs)) <= etol
    # values only
    m0, _ = op.predict(torch.tensor(alpha, device="cuda"), torch.tensor(Xs, device="cuda"),
                       with_grad=False)
    assert np.array_equal(m0.cpu().numpy(), mean.cpu().numpy()[:len(Xs)])
    op.close()


@pytest.mark.parametrize("make,rank", [(lambda: W.sine2d(), 20),
                                        (lambda: W.small3d(40, m=9, seed=3), 25)],
                         ids=["sine2d-gridform", "3d-q1form"])
def test_variance_estimate_matches_oracle(make, rank):
    need_gpu()
    from oracle.predict import variance_estimate, variance_dski
    from oracle.solve import QRPreconditioner, pivoted_cholesky
    p = make()
    orc = oracle_op(p)
    op = gpu_op(p, "fp64")
    pc = op.pivchol(rank)
    _, piv = pc.export()
    L, _, _ = pivoted_cholesky(orc.kgrad_diag(), orc.kgrad_row, rank, pivots=piv)
    Xs = _test_points(p, 70, 12)   # two batches of test points
    want = variance_estimate(orc, Xs, QRPreconditioner(L, orc.noise))
    _, var = op.predict(None, torch.tensor(Xs, device="cuda"), pc=pc)
    got = var.cpu().numpy()
    assert rel(got, want) <= 1e-9, rel(got, want)
    # the estimate lies below the D-SKI variance (M <= K~)
    if orc.N <= 3000:
        assert np.all(got <= variance_dski(orc, Xs) + 1e-10)
    pc.close()
    op.close()


def test_out_of_grid_test_point_is_reported():
    need_gpu()
    from paper_1810_12283_gb300 import DskiError
    p = W.sine2d()
    op = gpu_op(p, "fp64")
    alpha = torch.zeros(op.N, device="cuda", dtype=torch.float64)
    Xs = torch.tensor([[0.5, 0.5], [5.0, 0.5]], device="cuda", dtype=torch.float64)
    with pytest.raises(DskiError) as e:
        op.predict(alpha, Xs)
    assert "OUT_OF_GRID" in str(e.value)
    op.close()


def test_control_variate_variance_matches_oracle():
    """Sec. 5's randomized variance with the preconditioner estimate as
    control variate: with the same SplitMix64 probes the GPU equals the
    oracle (exact dense solves) to the PCG tolerance's effect, and it moves
    the preconditioner estimate toward the D-SKI variance."""
    need_gpu()
    from oracle.predict import variance_cv, variance_dski, variance_estimate
    from oracle.probes import rademacher
    from oracle.solve import QRPreconditioner, pivoted_cholesky
    p = W.small2d(300, m=24, seed=4, nv=1e-2, ng=1e-2)
    orc = oracle_op(p)
    op = gpu_op(p, "fp64")
    pc = op.pivchol(12)
    _, piv = pc.export()
    L, _, _ = pivoted_cholesky(orc.kgrad_diag(), orc.kgrad_row, 12, pivots=piv)
    Pc = QRPreconditioner(L, orc.noise)
    Xs = _test_points(p, 40, 13)
    P, seed = 64, 99
    got = op.predict_variance_cv(torch.tensor(Xs, device="cuda"), pc, probes=P, seed=seed,
                                 rtol=1e-11, maxit=20000).cpu().numpy()
    want = variance_cv(orc, Xs, Pc, rademacher(seed, len(Xs), P))
    assert np.max(np.abs(got - want)) <= 1e-9, np.max(np.abs(got - want))
    exact = variance_dski(orc, Xs)
    vhat = variance_estimate(orc, Xs, Pc)
    assert np.mean(np.abs(got - exact)) < np.mean(np.abs(vhat - exact))
    pc.close()
    op.close()
