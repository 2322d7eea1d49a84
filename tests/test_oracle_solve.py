"""Pins of the oracle solvers (Sec. 2, Sec. 3.3): the direct method, the
truncated pivoted Cholesky (exact at full rank, greedy pivots, Schur-complement
residual), the QR-form preconditioner against a dense inverse, and PCG against
the direct solve."""
import numpy as np

from oracle.dski import DSKI, Grid
from oracle.solve import chol_solve, chol_logdet, pivoted_cholesky, QRPreconditioner, pcg


def _op(n=50, seed=0, noise=(1e-3, 2e-3), m=16, ell=(0.25, 0.3)):
    X = np.random.default_rng(seed).uniform(0, 1, (n, 2))
    g = Grid(m=(m, m), lo=(-0.2, -0.2), hi=(1.2, 1.2))
    return DSKI(X, g, list(ell), 1.0, *noise)


def test_direct_method():
    op = _op()
    A = op.dense()
    b = np.random.default_rng(1).normal(size=op.N)
    x = chol_solve(A, b)
    # backward error of a backward-stable Cholesky solve
    assert np.linalg.norm(A @ x - b) / (np.linalg.norm(A, 2) * np.linalg.norm(x)) < 1e-14
    assert abs(chol_logdet(A) - np.linalg.slogdet(A)[1]) < 1e-9 * abs(np.linalg.slogdet(A)[1])


def test_pivoted_cholesky_full_rank_is_exact_and_greedy():
    rng = np.random.default_rng(2)
    F = rng.normal(size=(9, 6))
    A = F @ F.T                                   # rank 6 PSD
    L, piv, before = pivoted_cholesky(np.diag(A), lambda j: A[j], 9, rel_tol=1e-14)
    assert len(piv) == 6
    assert np.allclose(L @ L.T, A, atol=1e-11)
    for k, j in enumerate(piv):                   # greedy: pivot is the largest residual
        assert before[k][j] == before[k].max()
    # L restricted to pivot rows is lower triangular in pivot order
    assert np.allclose(np.triu(L[piv], 1), 0.0, atol=1e-13)


def test_pivoted_cholesky_residual_is_schur_complement():
    op = _op(n=20, seed=3)
    K = op.dense_kgrad()
    L, piv, _ = pivoted_cholesky(op.kgrad_diag(), op.kgrad_row, 7)
    S = K - L @ L.T
    P = np.array(piv)
    assert np.allclose(S[np.ix_(P, P)], 0.0, atol=1e-9 * np.abs(K).max())
    lam = np.linalg.eigvalsh(S)
    assert lam.min() > -1e-9 * np.abs(K).max()   # residual stays PSD


def test_qr_preconditioner_matches_dense_inverse():
    op = _op(n=40, seed=4)
    L, _, _ = pivoted_cholesky(op.kgrad_diag(), op.kgrad_row, 15)
    Pc = QRPreconditioner(L, op.noise)
    M = np.diag(op.noise) + L @ L.T
    b = np.random.default_rng(5).normal(size=(op.N, 3))
    want = np.linalg.solve(M, b)
    got = Pc.solve(b)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-10 * np.linalg.cond(M) ** 0.5
    assert abs(Pc.logdet() - np.linalg.slogdet(M)[1]) < 1e-9 * abs(np.linalg.slogdet(M)[1])
    C = Pc.sqrt_apply(np.eye(op.N))
    Cs = C / np.sqrt(op.noise)[:, None]          # D^{-1/2} C is the principal root: symmetric
    assert np.allclose(Cs, Cs.T, atol=1e-10 * np.abs(Cs).max())
    assert np.allclose(C @ C.T, M, rtol=0, atol=1e-10 * np.abs(M).max())


def test_pcg_matches_direct_and_preconditioning_helps():
    op = _op(n=80, seed=6)
    A = op.dense()
    b = np.random.default_rng(7).normal(size=op.N)
    x_ref = chol_solve(A, b)
    L, _, _ = pivoted_cholesky(op.kgrad_diag(), op.kgrad_row, 30)
    Pc = QRPreconditioner(L, op.noise)
    run = pcg(op.mvm, b, Pc.solve, rtol=1e-10, maxit=5000)
    assert run["relres"] < 2e-10
    assert np.linalg.norm(A @ (run["x"] - x_ref)) / np.linalg.norm(b) < 2e-10
    plain = pcg(op.mvm, b, None, rtol=1e-10, maxit=5000)
    assert run["iters"] < plain["iters"]
