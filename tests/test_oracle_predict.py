"""Pins of oracle.predict: the D-SKI mean against the exact GP mean on a
refining grid, interpolation of the data, the dense-solve variance against
its definition, and the preconditioner estimate's side of it (M <= K~, so
v_hat <= v)."""
import numpy as np

from oracle.dski import DSKI, Grid
from oracle.dse import dse_matrix
from oracle.predict import (dski_mean, exact_mean, variance_dski, variance_estimate)
from oracle.solve import QRPreconditioner, pivoted_cholesky


def _data(n=30, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, (n, 2))
    f = np.sin(2 * np.pi * X[:, 0]) * np.cos(2 * np.pi * X[:, 1])
    g1 = 2 * np.pi * np.cos(2 * np.pi * X[:, 0]) * np.cos(2 * np.pi * X[:, 1])
    g2 = -2 * np.pi * np.sin(2 * np.pi * X[:, 0]) * np.sin(2 * np.pi * X[:, 1])
    return X, np.concatenate([f, g1, g2])


def test_dski_mean_converges_to_the_exact_mean():
    X, y = _data()
    Xs = np.random.default_rng(1).uniform(0.1, 0.9, (7, 2))
    ell, sf, nz = 0.3, 1.0, 1e-4
    noise = np.full(y.size, nz)
    ref = exact_mean(X, y, Xs, [ell, ell], sf, noise)
    errs = []
    for m in (24, 48, 96):
        op = DSKI(X, Grid((m, m), (-0.15, -0.15), (1.15, 1.15)), [ell, ell], sf, nz, nz)
        alpha = np.linalg.solve(op.dense(), y)
        errs.append(np.max(np.abs(dski_mean(op, alpha, Xs) - ref)) / np.max(np.abs(ref)))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 2e-3, errs


def test_exact_mean_interpolates_at_small_noise():
    X, y = _data(12, seed=3)
    m = exact_mean(X, y, X, [0.3, 0.3], 1.0, np.full(y.size, 1e-10))
    assert np.max(np.abs(m - y)) <= 1e-5 * np.max(np.abs(y))


def test_exact_mean_blocks_match_the_derivative_kernel():
    # the test/train block of the stacked matrix is the mixed-argument block
    # of K^grad: with X* = X it reproduces K^grad K^grad~^{-1} y
    X, y = _data(9, seed=4)
    K = dse_matrix(X, [0.3, 0.3], 1.0)
    noise = np.full(y.size, 1e-3)
    want = K @ np.linalg.solve(K + np.diag(noise), y)
    got = exact_mean(X, y, X, [0.3, 0.3], 1.0, noise)
    assert np.allclose(got, want, rtol=1e-10, atol=1e-12)


def test_variance_estimate_brackets_and_full_rank_equality():
    X, y = _data(25, seed=5)
    op = DSKI(X, Grid((32, 32), (-0.15, -0.15), (1.15, 1.15)), [0.3, 0.3], 1.0, 1e-3, 1e-3)
    Xs = np.random.default_rng(6).uniform(0.1, 0.9, (6, 2))
    v = variance_dski(op, Xs)
    assert np.all(v > 0)
    Kg = op.dense_kgrad()
    diag, row = np.diag(Kg).copy(), (lambda j: Kg[:, j])
    for rank in (5, 20):
        L, _, _ = pivoted_cholesky(diag, row, rank)
        vh = variance_estimate(op, Xs, QRPreconditioner(L, op.noise))
        # M = D + L L^T <= K~ (the pivoted Cholesky residual is PSD), so
        # M^-1 >= K~^-1 and the estimate lies below the variance
        assert np.all(vh <= v + 1e-12), (rank, vh - v)
    # at full rank M = K~ and the estimate is the variance
    L, _, _ = pivoted_cholesky(diag, row, op.N)
    vh = variance_estimate(op, Xs, QRPreconditioner(L, op.noise))
    assert np.allclose(vh, v, rtol=1e-6, atol=1e-10)


def test_control_variate_estimator_is_exact_with_hadamard_probes():
    # with the n* columns of a Hadamard matrix as probes, sum_j z_j z_j^T = P I,
    # so the diagonal estimator is exact and v equals the D-SKI variance
    from scipy.linalg import hadamard
    from oracle.predict import variance_cv
    X, y = _data(25, seed=5)
    op = DSKI(X, Grid((32, 32), (-0.15, -0.15), (1.15, 1.15)), [0.3, 0.3], 1.0, 1e-3, 1e-3)
    Xs = np.random.default_rng(6).uniform(0.1, 0.9, (8, 2))
    Kg = op.dense_kgrad()
    L, _, _ = pivoted_cholesky(np.diag(Kg).copy(), lambda j: Kg[:, j], 10)
    Pc = QRPreconditioner(L, op.noise)
    H = hadamard(8).astype(np.float64)
    v = variance_cv(op, Xs, Pc, H)
    want = variance_dski(op, Xs)
    # v ~ 1e-4 is the difference of O(1) terms evaluated through K~^-1
    # (kappa ~ 1e6): rounding shows at ~1e-16 kappa ~ 1e-10 absolute
    assert np.allclose(v, want, rtol=0.0, atol=1e-9), (v, want)
    # Rademacher probes: unbiased, within the estimator's spread
    from oracle.probes import rademacher
    Z = rademacher(123, 8, 4000)
    vr = variance_cv(op, Xs, Pc, Z)
    assert np.all(np.abs(vr - want) <= 0.1 * np.abs(variance_estimate(op, Xs, Pc) - want) + 1e-9)
