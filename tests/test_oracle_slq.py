"""Pins of the SLQ oracle (Sec. 2): the Lanczos tridiagonal recovered from CG
coefficients equals explicit Lanczos; with full depth and scaled basis probes
the estimate is the exact log determinant; Rademacher estimates fall within
a few standard errors; the probe generator is the SplitMix64 stream."""
import numpy as np

from oracle.dski import DSKI, Grid
from oracle.solve import pivoted_cholesky, QRPreconditioner, pcg, chol_logdet
from oracle.slq import (lanczos_T_from_cg, lanczos_full, slq_logdet, quadrature_logdet_term,
                        slq_logdet_z)
from oracle.probes import splitmix64_stream, splitmix64_at, rademacher, preconditioned_probes


def _op(n, seed, m=12):
    X = np.random.default_rng(seed).uniform(0, 1, (n, 2))
    g = Grid(m=(m, m), lo=(-0.25, -0.25), hi=(1.25, 1.25))
    return DSKI(X, g, [0.3, 0.35], 1.0, 1e-2, 3e-2)


def test_T_from_cg_equals_explicit_lanczos():
    op = _op(12, 0)
    A = op.dense()
    b = np.random.default_rng(1).normal(size=op.N)
    k = 8
    run = pcg(op.mvm, b, None, rtol=0.0, maxit=k, record=k)
    d1, o1 = lanczos_T_from_cg(run["alphas"], run["betas"])
    d2, o2 = lanczos_full(A, b, k)
    assert np.allclose(d1, d2, rtol=1e-8)
    assert np.allclose(o1, np.abs(o2), rtol=1e-8)


def test_full_depth_basis_probes_give_exact_logdet():
    op = _op(4, 2, m=8)               # N = 12
    A = op.dense()
    L, _, _ = pivoted_cholesky(op.kgrad_diag(), op.kgrad_row, 3)
    Pc = QRPreconditioner(L, op.noise)
    W = np.sqrt(op.N) * np.eye(op.N)   # (1/N) sum w w^T = I
    est, _, _, _ = slq_logdet(op.mvm, Pc, W, depth=op.N, rtol=1e-14)
    assert abs(est - chol_logdet(A)) < 1e-8 * abs(chol_logdet(A))


def test_rademacher_estimate_within_standard_errors():
    op = _op(30, 3)
    A = op.dense()
    L, _, _ = pivoted_cholesky(op.kgrad_diag(), op.kgrad_row, 10)
    Pc = QRPreconditioner(L, op.noise)
    W = rademacher(77, op.N, 24)
    est, se, _, _ = slq_logdet(op.mvm, Pc, W, depth=30)
    assert abs(est - chol_logdet(A)) < 4 * se + 1e-6 * abs(chol_logdet(A))


def test_quadrature_of_diagonal_matrix():
    # T diagonal (off = 0): e1^T log(T) e1 = log T[0, 0]
    assert abs(quadrature_logdet_term(np.array([2.0, 5.0]), np.array([0.0]), 3.0) - 3 * np.log(2)) < 1e-14


def test_splitmix_counter_equals_stream_and_rademacher_layout():
    seed = 0x1234ABCD5678
    s = splitmix64_stream(seed, 50)
    assert all(splitmix64_at(seed, k + 1) == s[k] for k in range(50))
    N, P = 7, 3
    Z = rademacher(seed, N, P)
    for j in range(P):
        for e in range(N):
            bit = splitmix64_at(seed, j * N + e + 1) >> 63
            assert Z[e, j] == (1.0 if bit == 0 else -1.0)
    big = rademacher(5, 4000, 5)
    assert set(np.unique(big)) == {-1.0, 1.0}
    assert abs(big.mean()) < 0.03


def test_factor_probes_square_to_the_preconditioner():
    """C = [D^1/2, L] satisfies C C^T = M, and the probe generator is C w."""
    op = _op(10, 5)
    L, _, _ = pivoted_cholesky(op.kgrad_diag(), op.kgrad_row, 6)
    Pc = QRPreconditioner(L, op.noise)
    C = Pc.factor_apply(np.eye(op.N + 6))
    assert np.allclose(C @ C.T, np.diag(op.noise) + L @ L.T, rtol=0, atol=1e-13)
    Z = preconditioned_probes(99, Pc, 3)
    assert np.allclose(Z, C @ rademacher(99, op.N + 6, 3), rtol=0, atol=1e-14)


def test_full_depth_factor_basis_probes_give_exact_logdet():
    """Probes sqrt(P) C e_i (i < P = N + r) average z z^T to M exactly, so at
    full Lanczos depth the preconditioned estimator is the exact log det."""
    op = _op(4, 6, m=8)               # N = 12
    A = op.dense()
    L, _, _ = pivoted_cholesky(op.kgrad_diag(), op.kgrad_row, 3)
    Pc = QRPreconditioner(L, op.noise)
    P = op.N + 3
    Z = np.sqrt(P) * Pc.factor_apply(np.eye(P))
    est, _, _, _ = slq_logdet_z(op.mvm, Pc, Z, depth=op.N, rtol=1e-14)
    assert abs(est - chol_logdet(A)) < 1e-8 * abs(chol_logdet(A))


def test_preconditioned_rademacher_within_standard_errors():
    op = _op(30, 7)
    A = op.dense()
    L, _, _ = pivoted_cholesky(op.kgrad_diag(), op.kgrad_row, 10)
    Pc = QRPreconditioner(L, op.noise)
    est, se, _, _ = slq_logdet_z(op.mvm, Pc, preconditioned_probes(5, Pc, 24), depth=30)
    assert abs(est - chol_logdet(A)) < 4 * se + 1e-6 * abs(chol_logdet(A))


def test_splitmix64_matches_published_reference_outputs():
    """Pin the generator itself (not only its two forms against each other):
    the first outputs of the stream for two seeds are the values published
    with the reference implementation (tests/golden/splitmix64.txt).  A wrong
    constant in the increment or the finaliser changes every one of them."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")
    rows = [list(map(int, ln.split())) for ln in open(path)
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 2
    for seed, *expected in rows:
        assert splitmix64_stream(seed, len(expected)) == expected
        assert [splitmix64_at(seed, k + 1) for k in range(len(expected))] == expected
        # the vectorised form used to build probe matrices: sign of the top bit
        Z = rademacher(seed, len(expected), 1)[:, 0]
        assert list(Z) == [1.0 if v >> 63 == 0 else -1.0 for v in expected]
