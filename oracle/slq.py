"""Stochastic Lanczos quadrature for log|K~| (Sec. 2: log|K~| = tr(log K~)
estimated with probe vectors and the Lanczos / Gauss-quadrature connection).

Preconditioned form (a reading: the paper does not say how SLQ combines with
the Sec. 3.3 preconditioner).  With M = C C^T,
  log|K~| = log|M| + tr log(C^{-1} K~ C^{-T}).
PCG on K~ x = C w with preconditioner M runs, in exact arithmetic, the
Lanczos process of A_hat = C^{-1} K~ C^{-T} started at w/||w||, and its
coefficients give the Lanczos tridiagonal (Saad, Iterative Methods for
Sparse Linear Systems, 2nd ed., Sec. 6.7.3):
  T[j, j]   = 1/alpha_j + beta_{j-1}/alpha_{j-1}   (second term absent for j = 0)
  T[j, j+1] = sqrt(beta_j) / alpha_j
Gauss quadrature: w^T log(A_hat) w ~ ||w||^2 sum_j tau_{1j}^2 log(lambda_j)
with (lambda_j, tau_j) the eigenpairs of T.  The Hutchinson estimate of the
trace is the mean over probes.

Test infrastructure only (see ``oracle/__init__``).
"""
import numpy as np
import scipy.linalg as sla


def lanczos_T_from_cg(alphas, betas):
    """Tridiagonal T_k from k CG steps (alphas[0..k-1], betas[0..k-2] used)."""
    k = len(alphas)
    diag = np.empty(k)
    off = np.empty(max(k - 1, 0))
    for j in range(k):
        diag[j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j < k - 1:
            off[j] = np.sqrt(betas[j]) / alphas[j]
    return diag, off


def lanczos_full(A, q0, k):
    """Plain Lanczos with full reorthogonalisation on a dense symmetric A,
    k steps from q0; returns the tridiagonal (diag, off)."""
    N = A.shape[0]
    Q = np.zeros((N, k))
    q = q0 / np.linalg.norm(q0)
    diag, off = [], []
    beta = 0.0
    qprev = np.zeros(N)
    for j in range(k):
        Q[:, j] = q
        v = A @ q - beta * qprev
        a = q @ v
        v = v - a * q
        v = v - Q[:, :j + 1] @ (Q[:, :j + 1].T @ v)
        diag.append(a)
        beta = np.linalg.norm(v)
        if j < k - 1:
            off.append(beta)
        qprev, q = q, v / beta
    return np.array(diag), np.array(off)


def quadrature_logdet_term(diag, off, znorm2):
    """||z||^2 * e1^T log(T) e1 by the eigen-decomposition of T (Golub-Welsch)."""
    lam, vec = sla.eigh_tridiagonal(diag, off)
    return znorm2 * np.sum(vec[0, :] ** 2 * np.log(lam))


def slq_logdet(mvm, precond, probes, depth, rtol=1e-12, maxit=10000):
    """Preconditioned SLQ estimate of log|K~| from Rademacher probes w (N x P).

    ``precond`` is an oracle.solve.QRPreconditioner (M = D + L L^T); each
    probe runs PCG on K~ x = C w.  Returns (estimate, standard error, per-probe
    terms, per-probe PCG results).
    """
    from .solve import pcg
    P = probes.shape[1]
    terms, runs = [], []
    for j in range(P):
        w = probes[:, j]
        run = pcg(mvm, precond.sqrt_apply(w), precond.solve, rtol=rtol, maxit=maxit,
                  record=depth)
        k = min(depth, run["iters"])
        dg, of = lanczos_T_from_cg(run["alphas"][:k], run["betas"][:k])
        terms.append(quadrature_logdet_term(dg, of, w @ w))
        runs.append(run)
    terms = np.array(terms)
    est = precond.logdet() + terms.mean()
    se = terms.std(ddof=1) / np.sqrt(P) if P > 1 else float("nan")
    return est, se, terms, runs


def slq_logdet_z(mvm, precond, Z, depth, rtol=1e-12, maxit=10000):
    """Preconditioned SLQ from probe vectors z_j (columns of Z) with
    E[z z^T] = M.  For such z, E[z^T M^{-1/2} log(A_hat) M^{-1/2} z] =
    tr log(A_hat), A_hat = M^{-1/2} K~ M^{-1/2}; PCG on K~ x = z is the
    Lanczos process on A_hat from M^{-1/2} z, whose squared norm is
    z^T M^{-1} z, so the quadrature term of probe j is
    (z_j^T M^{-1} z_j) e1^T log(T_j) e1.  Returns (estimate, standard error,
    per-probe terms, per-probe PCG results)."""
    from .solve import pcg
    P = Z.shape[1]
    terms, runs = [], []
    for j in range(P):
        z = Z[:, j]
        run = pcg(mvm, z, precond.solve, rtol=rtol, maxit=maxit, record=depth)
        k = min(depth, run["iters"])
        dg, of = lanczos_T_from_cg(run["alphas"][:k], run["betas"][:k])
        terms.append(quadrature_logdet_term(dg, of, z @ precond.solve(z)))
        runs.append(run)
    terms = np.array(terms)
    est = precond.logdet() + terms.mean()
    se = terms.std(ddof=1) / np.sqrt(P) if P > 1 else float("nan")
    return est, se, terms, runs
