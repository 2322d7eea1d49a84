"""Solvers of Sec. 2 and Sec. 3.3, written out plainly in FP64.

* Direct method (Sec. 2, after Eq. 1): Cholesky of K~ for solves and log det.
* Truncated pivoted Cholesky (Sec. 3.3, following Harbrecht et al. 2012):
  greedy pivot = argmax of the residual diagonal; each step needs only the
  diagonal and the pivot row.  K^grad ~ (Pi L)(Pi L)^T.
* Preconditioner M = D + L L^T (Sec. 3.3 writes D = sigma^2 I) applied by the
  QR-stable formula instead of Sherman-Morrison-Woodbury:
  [D^{-1/2} L; I] = [Q1; Q2] R (economy QR), then
  M^{-1} b = D^{-1/2} (y - Q1 Q1^T y) with y = D^{-1/2} b.
  For D = sigma^2 I this is the paper's sigma^-2 (b - Q1 Q1^T b).
* Preconditioned conjugate gradients (Sec. 2 "conjugate gradients", Sec. 3.3).

Test infrastructure only (see ``oracle/__init__``).
"""
import numpy as np
import scipy.linalg as sla


def chol_solve(A, b):
    """x = A^{-1} b via Cholesky (the O(n^3) direct method of Sec. 2)."""
    cf = sla.cho_factor(A, lower=True)
    return sla.cho_solve(cf, b)


def chol_logdet(A):
    """log|A| = 2 sum log diag(chol(A))."""
    Lc = np.linalg.cholesky(A)
    return 2.0 * np.sum(np.log(np.diag(Lc)))


def pivoted_cholesky(diag, row, rank, rel_tol=0.0, pivots=None):
    """Truncated pivoted Cholesky of a PSD matrix given only its diagonal and
    a row callback (Sec. 3.3).

    Step k: j = argmax of the residual diagonal (lowest index on ties), stop
    if the residual trace <= rel_tol * initial trace or the pivot is <= 0;
    L[:, k] = (row(j) - L[:, :k] L[j, :k]^T) / sqrt(res[j]);
    res -= L[:, k]^2.

    ``pivots`` forces a given pivot sequence (used to compare against a
    solver whose arithmetic broke a near-tie differently).
    Returns (L[:, :rank_achieved], pivot list, residual-diagonal list
    before each step).
    """
    res = np.array(diag, dtype=np.float64, copy=True)
    N = res.shape[0]
    tr0 = res.sum()
    L = np.zeros((N, rank))
    piv, before = [], []
    for k in range(rank):
        if res.sum() <= rel_tol * tr0:
            break
        j = int(np.argmax(res)) if pivots is None else int(pivots[k])
        if res[j] <= 0.0:
            break
        before.append(res.copy())
        col = (np.asarray(row(j), np.float64) - L[:, :k] @ L[j, :k]) / np.sqrt(res[j])
        L[:, k] = col
        res = res - col**2
        piv.append(j)
    return L[:, :len(piv)], piv, before


class QRPreconditioner:
    """M = D + L L^T applied through the economy QR of [D^{-1/2} L; I] (Sec. 3.3)."""

    def __init__(self, L, Ddiag):
        self.L = np.asarray(L, np.float64)
        self.D = np.asarray(Ddiag, np.float64)
        N, r = self.L.shape
        Lt = self.L / np.sqrt(self.D)[:, None]
        Q, R = np.linalg.qr(np.vstack([Lt, np.eye(r)]), mode="reduced")
        self.Q1 = Q[:N]
        self.Lt = Lt

    def solve(self, b):
        """M^{-1} b = D^{-1/2} (y - Q1 (Q1^T y)), y = D^{-1/2} b."""
        b = np.asarray(b, np.float64)
        sq = np.sqrt(self.D) if b.ndim == 1 else np.sqrt(self.D)[:, None]
        y = b / sq
        return (y - self.Q1 @ (self.Q1.T @ y)) / sq

    def logdet(self):
        """log|M| = sum log D + log|I + Lt^T Lt| (Sylvester's determinant identity)."""
        r = self.Lt.shape[1]
        return np.sum(np.log(self.D)) + np.linalg.slogdet(np.eye(r) + self.Lt.T @ self.Lt)[1]

    def factor_apply(self, w):
        """C w with the rectangular factor C = [D^{1/2}, L] (N x (N + r)), so
        that C C^T = D + L L^T = M: w stacks an N-vector w1 over an r-vector
        w2 and C w = D^{1/2} w1 + L w2."""
        w = np.asarray(w, np.float64)
        N, r = self.L.shape
        sq = np.sqrt(self.D) if w.ndim == 1 else np.sqrt(self.D)[:, None]
        return sq * w[:N] + self.L @ w[N:]

    def sqrt_apply(self, w):
        """C w with C C^T = M, C = D^{1/2} (I + Lt Lt^T)^{1/2} (principal square
        root via the thin SVD Lt = U S V^T: I + U (sqrt(1 + S^2) - 1) U^T)."""
        w = np.asarray(w, np.float64)
        U, S, _ = np.linalg.svd(self.Lt, full_matrices=False)
        core = np.sqrt(1.0 + S**2) - 1.0
        if w.ndim == 1:
            return np.sqrt(self.D) * (w + U @ (core * (U.T @ w)))
        return np.sqrt(self.D)[:, None] * (w + U @ (core[:, None] * (U.T @ w)))


def pcg(mvm, b, precond=None, rtol=1e-10, maxit=1000, x0=None, record=0):
    """Preconditioned CG for one right-hand side.

    Stops when the recursive residual satisfies ||r|| <= rtol ||b||.
    Returns dict(x, iters, relres (true residual), alphas, betas) where
    alphas/betas are the first ``record`` CG coefficients
    (beta_k = r_{k+1}^T z_{k+1} / r_k^T z_k).
    """
    b = np.asarray(b, np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64)
    Minv = (lambda v: v) if precond is None else precond
    r = b - mvm(x) if x0 is not None else b.copy()
    z = Minv(r)
    p = z.copy()
    rz = r @ z
    bn = np.linalg.norm(b)
    alphas, betas = [], []
    it = 0
    if bn == 0.0:
        return dict(x=x, iters=0, relres=0.0, alphas=alphas, betas=betas)
    while np.linalg.norm(r) > rtol * bn and it < maxit:
        q = mvm(p)
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        z = Minv(r)
        rz_new = r @ z
        beta = rz_new / rz
        if it < record:
            alphas.append(alpha)
            betas.append(beta)
        p = z + beta * p
        rz = rz_new
        it += 1
    relres = np.linalg.norm(b - mvm(x)) / bn
    return dict(x=x, iters=it, relres=relres, alphas=alphas, betas=betas)
