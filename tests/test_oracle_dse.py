"""Pins of the exact derivative SE kernel (Sec. 2, App. A, App. B):
finite differences of the kernel value, a hand-evaluated d = 1 case,
symmetry and positive semi-definiteness."""
import numpy as np

from oracle.dse import se_kernel, dse_matrix


def _fd_blocks(X, ell, sf, i, j, h=1e-5):
    d = X.shape[1]
    k = lambda a, b: se_kernel(a, b, ell, sf)
    xi, xj = X[i], X[j]
    E = np.eye(d) * h
    g1 = np.array([(k(xi + E[p], xj) - k(xi - E[p], xj)) / (2 * h) for p in range(d)])
    g2 = np.array([(k(xi, xj + E[q]) - k(xi, xj - E[q])) / (2 * h) for q in range(d)])
    H = np.array([[(k(xi + E[p], xj + E[q]) - k(xi + E[p], xj - E[q])
                    - k(xi - E[p], xj + E[q]) + k(xi - E[p], xj - E[q])) / (4 * h * h)
                   for q in range(d)] for p in range(d)])
    return g1, g2, H


def test_blocks_match_finite_differences():
    rng = np.random.default_rng(1)
    n, d = 5, 3
    X = rng.uniform(0, 1, (n, d))
    ell = np.array([0.4, 0.7, 0.55])
    sf = 1.3
    K = dse_matrix(X, ell, sf)
    for i in range(n):
        for j in range(n):
            g1, g2, H = _fd_blocks(X, ell, sf, i, j)
            assert abs(K[i, j] - se_kernel(X[i], X[j], ell, sf)) < 1e-15
            for p in range(d):
                assert abs(K[(p + 1) * n + i, j] - g1[p]) < 1e-7       # d/dx_i,p (first argument)
                assert abs(K[i, (p + 1) * n + j] - g2[p]) < 1e-7       # d/dx_j,p (second argument)
                for q in range(d):
                    assert abs(K[(p + 1) * n + i, (q + 1) * n + j] - H[p, q]) < 2e-5


def test_hand_evaluated_d1_pair():
    # x0 = 0, x1 = 1, l = 1, s_f = 1; order [v0, v1, g0, g1]
    e = np.exp(-0.5)
    want = np.array([[1, e, 0, -e],
                     [e, 1, e, 0],
                     [0, e, 1, 0],
                     [-e, 0, 0, 1]])
    # entry (g0, v1) = dk(x0, x1)/dx0 = -(x0 - x1) k = +e;  (v0, g1) = dk/dx1 = (x0 - x1) k = -e
    # entry (g0, g1) = (1 - (x0 - x1)^2) k = 0
    K = dse_matrix(np.array([[0.0], [1.0]]), [1.0], 1.0)
    assert np.allclose(K, want, atol=1e-15)


def test_symmetric_psd():
    rng = np.random.default_rng(2)
    X = rng.uniform(0, 1, (30, 2))
    K = dse_matrix(X, [0.3, 0.2], 0.9)
    assert np.allclose(K, K.T, atol=1e-14)
    lam = np.linalg.eigvalsh(K)
    assert lam.min() >= -1e-12 * lam.max()
