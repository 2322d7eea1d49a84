"""Prediction with the D-SKI GP: mean, gradient and the pivoted-Cholesky
variance estimate (Sec. 5, prediction for Bayesian optimisation).

* Mean and gradient at test points X*: the cross-covariance between the
  test values / gradients and the training data is approximated the same
  way as K^grad (Sec. 3.1), K(X*, X)^grad ~ B* K_UU B^T with
  B* = [W*; dW*_1; ...] the interpolation rows of the test points, so
      mu* = B* K_UU B^T alpha,   alpha = K~^{-1} y.
* Variance: v(x) = k(x, x) - k_x^T K~^{-1} k_x with k_x = B K_UU w*(x)^T;
  the fast estimate of Sec. 5 replaces K~^{-1} by the preconditioner solve
  M^{-1}, M = D + L L^T the pivoted Cholesky approximation (Sec. 3.3):
      v_hat(x) = k(x, x) - k_x^T M^{-1} k_x,   k(x, x) = s_f^2.
  (For equal noise s^2 this is the text's s^-2 (|k_x|^2 - |Q1^T k_x|^2).)

Test infrastructure only (see ``oracle/__init__``).
"""
import numpy as np

from .dski import interp_matrix, kuu_apply
from .dse import dse_matrix


def dski_mean(op, alpha, Xs):
    """mu* = B* K_UU B^T alpha for the D-SKI operator `op` (oracle.dski.DSKI):
    block order [values (n*); d/dx_1 (n*); ...]."""
    Bs = interp_matrix(Xs, op.grid)
    g = op.B.T @ np.asarray(alpha, np.float64)
    h = kuu_apply(op.grid, op.ell, op.sf, g[:, None])[:, 0]
    return Bs @ h


def dski_cross(op, Xs):
    """k_x for every test point: the N x n* matrix B K_UU W*^T (value rows of
    the test interpolation only)."""
    Bs = interp_matrix(Xs, op.grid)
    ns = np.asarray(Xs).shape[0]
    Ws = Bs[:ns].toarray().T                       # m x n*
    return op.B @ kuu_apply(op.grid, op.ell, op.sf, Ws)


def variance_estimate(op, Xs, precond):
    """v_hat(x) = s_f^2 - k_x^T M^{-1} k_x with M^{-1} = precond.solve."""
    Kx = dski_cross(op, Xs)
    Z = precond.solve(Kx)
    return op.sf**2 - np.sum(Kx * Z, axis=0)


def variance_dski(op, Xs):
    """The D-SKI predictive variance s_f^2 - k_x^T K~^{-1} k_x, dense solve."""
    Kx = dski_cross(op, Xs)
    A = op.dense()
    return op.sf**2 - np.sum(Kx * np.linalg.solve(A, Kx), axis=0)


def exact_mean(X, y, Xs, lengthscale, outputscale, noise):
    """The exact GP-with-derivatives mean at X* (values and gradients), from
    the dense derivative SE matrix of the stacked points [X*; X]."""
    X = np.asarray(X, np.float64)
    Xs = np.asarray(Xs, np.float64)
    n, d = X.shape
    ns = Xs.shape[0]
    Kall = dse_matrix(np.vstack([Xs, X]), lengthscale, outputscale)
    tot = ns + n
    test_rows = np.concatenate([np.arange(ns) + c * tot for c in range(d + 1)])
    train_cols = np.concatenate([ns + np.arange(n) + c * tot for c in range(d + 1)])
    Kst = Kall[np.ix_(test_rows, train_cols)]
    Ktt = Kall[np.ix_(train_cols, train_cols)] + np.diag(noise)
    return Kst @ np.linalg.solve(Ktt, np.asarray(y, np.float64))


def variance_cv(op, Xs, precond, Z):
    """The randomized predictive variance of Sec. 5 with the preconditioner
    estimate as control variate:
        v = v_hat - diag(K_*X (K~^-1 - M^-1) K_X*),
        diag(A) ~ (1/P) sum_j z_j .* (A z_j)      (Bekas et al.'s estimator),
    for the probe columns Z (n* x P, entries +-1).  K_*X = K_X*^T for the
    value rows of the test points (oracle.predict.dski_cross)."""
    Kx = dski_cross(op, Xs)                        # N x n*
    U = Kx @ Z                                     # N x P
    A = np.linalg.solve(op.dense(), U)
    Bm = precond.solve(U)
    Wz = Kx.T @ (A - Bm)                           # n* x P
    return variance_estimate(op, Xs, precond) - np.mean(Z * Wz, axis=1)
