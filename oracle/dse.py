"""Exact derivative SE kernel matrix K^grad ("D-SE") -- Sec. 2 and App. A/B.

Block order of rows and columns: [values (n); d/dx_1 (n); ...; d/dx_d (n)],
the order of the D-SKI block matrix in Sec. 3.1.  For points x_i, x_j,
r = x_i - x_j and per-dimension length scales l (ARD form of App. A):

  k(x_i, x_j)             = s_f^2 exp(-sum_k r_k^2 / (2 l_k^2))
  d k / d x_{i,p}         = -r_p / l_p^2 * k           (first argument)
  d k / d x_{j,q}         = +r_q / l_q^2 * k           (second argument, App. B)
  d2 k / dx_{i,p} dx_{j,q} = (delta_pq / l_p^2 - r_p r_q / (l_p^2 l_q^2)) * k

The lower-left block of k^grad in Sec. 2 differentiates the first argument,
the upper-right block the second; App. B states the second-argument form.

Test infrastructure only (see ``oracle/__init__``).
"""
import numpy as np


def se_kernel(xi, xj, lengthscale, outputscale):
    """SE kernel value of App. A (ARD length scales)."""
    r = np.asarray(xi, np.float64) - np.asarray(xj, np.float64)
    ell = np.asarray(lengthscale, np.float64)
    return outputscale**2 * np.exp(-0.5 * np.sum((r / ell) ** 2))


def dse_matrix(X, lengthscale, outputscale):
    """Dense K^grad of size n(d+1) x n(d+1), built entry block by block."""
    X = np.asarray(X, np.float64)
    n, d = X.shape
    ell2 = np.asarray(lengthscale, np.float64) ** 2
    R = X[:, None, :] - X[None, :, :]                      # r_ij = x_i - x_j
    K = outputscale**2 * np.exp(-0.5 * np.sum(R**2 / ell2, axis=2))
    N = n * (d + 1)
    out = np.empty((N, N))
    out[:n, :n] = K
    for q in range(d):                                     # value row, d/dx_j,q column
        out[:n, (q + 1) * n:(q + 2) * n] = R[:, :, q] / ell2[q] * K
    for p in range(d):                                     # d/dx_i,p row, value column
        out[(p + 1) * n:(p + 2) * n, :n] = -R[:, :, p] / ell2[p] * K
    for p in range(d):
        for q in range(d):
            delta = 1.0 / ell2[p] if p == q else 0.0
            blk = (delta - R[:, :, p] * R[:, :, q] / (ell2[p] * ell2[q])) * K
            out[(p + 1) * n:(p + 2) * n, (q + 1) * n:(q + 2) * n] = blk
    return out
