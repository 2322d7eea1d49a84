"""Log marginal likelihood (Eq. 1) and its hyperparameter gradient.

With mu = 0 and N = n(d+1) observations (values and gradients):
  L(theta) = -1/2 [ y^T alpha + log|K~| + N log(2 pi) ],  alpha = K~^{-1} y,
  dL/dtheta = 1/2 alpha^T (dK~/dtheta) alpha - 1/2 tr(K~^{-1} dK~/dtheta).

theta = (log l_1, ..., log l_d, log s_f, log sigma_n).  In D-SKI the
interpolation matrix B does not depend on theta, so
  dK~/dlog l_k  = B (s_f^2 K_1 (x) .. (x) dK_k/dlog l_k (x) .. (x) K_d) B^T,
  dK_k/dlog l_k = K_k * (u_a - u_b)^2 / l_k^2,
  dK~/dlog s_f  = 2 B K_UU B^T,
  dK~/dlog sigma_n = 2 diag(noise)   (both noise levels scale with sigma_n^2).

Test infrastructure only (see ``oracle/__init__``).
"""
import numpy as np

from .dski import DSKI, dense_kgrad_factored, kfactor, kfactor_dlogell, kron_apply
from .solve import chol_solve, chol_logdet, pcg


def dtheta_mvm(op: DSKI, i, V):
    """(dK~/dtheta_i) V for theta index i (see the module docstring)."""
    d = op.d
    V = np.asarray(V, np.float64)
    V2 = V.reshape(op.N, -1)
    if i < d:
        facs = [kfactor_dlogell(op.grid, k, op.ell[k]) if k == i else kfactor(op.grid, k, op.ell[k])
                for k in range(d)]
        out = op.B @ (op.sf**2 * kron_apply(facs, op.B.T @ V2))
    elif i == d:
        out = 2.0 * op.kgrad_mvm(V2)
    else:
        out = 2.0 * op.noise[:, None] * V2
    return out.ravel() if V.ndim == 1 else out


def dtheta_dense_factored(op: DSKI, i):
    """dK~/dtheta_i as a dense matrix through dense_kgrad_factored (for grids
    too large for the dense K_UU); equals dtheta_mvm(op, i, I)."""
    d = op.d
    if i < d:
        facs = [kfactor_dlogell(op.grid, k, op.ell[k]) if k == i else kfactor(op.grid, k, op.ell[k])
                for k in range(d)]
        return dense_kgrad_factored(op.X, op.grid, facs, op.sf)
    if i == d:
        facs = [kfactor(op.grid, k, op.ell[k]) for k in range(d)]
        return 2.0 * dense_kgrad_factored(op.X, op.grid, facs, op.sf)
    return np.diag(2.0 * op.noise)


def _dense_matrix(op: DSKI, factored):
    if not factored:
        return op.dense()
    facs = [kfactor(op.grid, k, op.ell[k]) for k in range(op.d)]
    return dense_kgrad_factored(op.X, op.grid, facs, op.sf) + np.diag(op.noise)


def mll_dense(op: DSKI, y, factored=False):
    """Eq. 1 by the direct (Cholesky) method; factored=True forms K~ through
    dense_kgrad_factored (large grids)."""
    A = _dense_matrix(op, factored)
    alpha = chol_solve(A, y)
    return -0.5 * (y @ alpha + chol_logdet(A) + op.N * np.log(2.0 * np.pi))


def mll_grad_dense(op: DSKI, y, factored=False):
    """Exact gradient of Eq. 1 with the trace taken through the dense inverse."""
    A = _dense_matrix(op, factored)
    alpha = chol_solve(A, y)
    Ainv = chol_solve(A, np.eye(op.N))
    g = []
    for i in range(op.d + 2):
        dK = dtheta_dense_factored(op, i) if factored else dtheta_mvm(op, i, np.eye(op.N))
        g.append(0.5 * alpha @ dK @ alpha - 0.5 * np.sum(Ainv * dK.T))
    return np.array(g)


def mll_grad_hutchinson(op: DSKI, y, precond, probes, rtol=1e-12, maxit=20000):
    """Stochastic gradient with probes z_j = C w_j (E[z z^T] = M):
    tr(K~^{-1} dK~) ~ mean_j (K~^{-1} z_j)^T dK~ (M^{-1} z_j).

    Returns (data-fit part 1/2 alpha^T dK alpha, trace estimates, gradient).
    """
    run = pcg(op.mvm, y, precond.solve, rtol=rtol, maxit=maxit)
    alpha = run["x"]
    fit = np.array([0.5 * alpha @ dtheta_mvm(op, i, alpha) for i in range(op.d + 2)])
    P = probes.shape[1]
    tr = np.zeros(op.d + 2)
    for j in range(P):
        z = precond.sqrt_apply(probes[:, j])
        u = pcg(op.mvm, z, precond.solve, rtol=rtol, maxit=maxit)["x"]
        v = precond.solve(z)
        for i in range(op.d + 2):
            tr[i] += u @ dtheta_mvm(op, i, v)
    tr /= P
    return fit, tr, fit - 0.5 * tr


def mll_grad_hutchinson_z(op: DSKI, y, precond, Z, rtol=1e-12, maxit=20000):
    """As mll_grad_hutchinson with the probe vectors z_j (E[z z^T] = M)
    given directly: tr(K~^{-1} dK~) ~ mean_j (K~^{-1} z_j)^T dK~ (M^{-1} z_j)."""
    run = pcg(op.mvm, y, precond.solve, rtol=rtol, maxit=maxit)
    alpha = run["x"]
    fit = np.array([0.5 * alpha @ dtheta_mvm(op, i, alpha) for i in range(op.d + 2)])
    P = Z.shape[1]
    tr = np.zeros(op.d + 2)
    for j in range(P):
        z = Z[:, j]
        u = pcg(op.mvm, z, precond.solve, rtol=rtol, maxit=maxit)["x"]
        v = precond.solve(z)
        for i in range(op.d + 2):
            tr[i] += u @ dtheta_mvm(op, i, v)
    tr /= P
    return fit, tr, fit - 0.5 * tr


def mll_grad_hutchinson_direct(op: DSKI, y, precond, Z, factored=False):
    """The estimator of mll_grad_hutchinson_z with every solve taken from the
    Cholesky factor of the dense K~ instead of PCG (exact solves, for systems
    small enough to factor but slow to iterate on):
      fit_i = 1/2 a^T dK~_i a,  a = K~^{-1} y,
      tr_i  = mean_j (K~^{-1} z_j)^T dK~_i (M^{-1} z_j),
      grad_i = fit_i - 1/2 tr_i.
    factored=True forms K~ and dK~_i through dense_kgrad_factored."""
    A = _dense_matrix(op, factored)
    alpha = chol_solve(A, y)
    Z = np.asarray(Z, np.float64)
    U = chol_solve(A, Z)
    V = np.column_stack([precond.solve(Z[:, j]) for j in range(Z.shape[1])])
    fit = np.empty(op.d + 2)
    tr = np.empty(op.d + 2)
    for i in range(op.d + 2):
        if factored:
            dK = dtheta_dense_factored(op, i)
            fit[i] = 0.5 * alpha @ (dK @ alpha)
            tr[i] = np.mean(np.sum(U * (dK @ V), axis=0))
        else:
            fit[i] = 0.5 * alpha @ dtheta_mvm(op, i, alpha)
            tr[i] = np.mean(np.sum(U * dtheta_mvm(op, i, V), axis=0))
    return fit, tr, fit - 0.5 * tr
