"""Pins of the explicit D-SKI oracle (Sec. 3.1): interpolation identities,
dense-vs-Kronecker agreement, the congruence structure (symmetric PSD), the
diagonal/row callbacks, and convergence to the exact D-SE kernel as the grid
is refined."""
import numpy as np
import pytest

from oracle.dse import dse_matrix
from oracle.dski import DSKI, Grid, interp_matrix, kuu_dense, kuu_apply


def _pts(n, d, seed):
    return np.random.default_rng(seed).uniform(0, 1, (n, d))


@pytest.mark.parametrize("d", [1, 2, 3])
def test_rows_partition_of_unity(d):
    g = Grid(m=(12,) * d, lo=(-0.3,) * d, hi=(1.3,) * d)
    X = _pts(40, d, d)
    B = interp_matrix(X, g).toarray()
    n = X.shape[0]
    assert np.allclose(B[:n].sum(1), 1.0, atol=1e-13)
    assert np.allclose(B[n:].sum(1), 0.0, atol=1e-10)
    assert np.all((B[:n] != 0).sum(1) <= 4**d)


def test_reproduces_quadratic_fields_in_2d():
    g = Grid(m=(15, 18), lo=(-0.3, -0.25), hi=(1.3, 1.2))
    X = _pts(50, 2, 3)
    B = interp_matrix(X, g)
    u1 = g.nodes(0)[:, None] * np.ones(g.m[1])[None, :]
    u2 = np.ones(g.m[0])[:, None] * g.nodes(1)[None, :]
    f = lambda a, b: 0.3 + 1.1 * a - 0.7 * b + 0.9 * a * a - 1.3 * a * b + 0.4 * b * b
    fx = lambda a, b: 1.1 + 1.8 * a - 1.3 * b
    fy = lambda a, b: -0.7 - 1.3 * a + 0.8 * b
    vals = B @ f(u1, u2).ravel()
    n = X.shape[0]
    assert np.allclose(vals[:n], f(X[:, 0], X[:, 1]), atol=1e-12)
    assert np.allclose(vals[n:2 * n], fx(X[:, 0], X[:, 1]), atol=1e-9)
    assert np.allclose(vals[2 * n:], fy(X[:, 0], X[:, 1]), atol=1e-9)


def test_kronecker_apply_equals_dense():
    g = Grid(m=(7, 5, 6), lo=(0, -1, 0.5), hi=(1, 2, 1.5))
    ell = np.array([0.3, 0.9, 0.2])
    G = np.random.default_rng(4).normal(size=(g.size, 3))
    assert np.allclose(kuu_apply(g, ell, 1.7, G), kuu_dense(g, ell, 1.7) @ G, rtol=0, atol=1e-13)


def test_mvm_dense_symmetric_psd():
    g = Grid(m=(16, 16), lo=(-0.2, -0.2), hi=(1.2, 1.2))
    op = DSKI(_pts(60, 2, 5), g, [0.2, 0.3], 1.1, 1e-3, 2e-3)
    A = op.dense()
    V = np.random.default_rng(6).normal(size=(op.N, 2))
    assert np.allclose(op.mvm(V), A @ V, rtol=0, atol=1e-11 * np.abs(A).max())
    assert np.allclose(A, A.T, atol=1e-12 * np.abs(A).max())
    Kg = op.dense_kgrad()
    lam = np.linalg.eigvalsh(Kg)
    assert lam.min() >= -1e-11 * lam.max()        # congruence of PSD K_UU


def test_diag_and_row_callbacks():
    g = Grid(m=(12, 10, 11), lo=(-0.3,) * 3, hi=(1.3,) * 3)
    op = DSKI(_pts(15, 3, 7), g, [0.3, 0.4, 0.5], 0.8, 1e-2, 1e-2)
    Kg = op.dense_kgrad()
    assert np.allclose(op.kgrad_diag(), np.diag(Kg), rtol=1e-12, atol=0)
    for j in [0, 7, 16, 31, 59]:
        assert np.allclose(op.kgrad_row(j), Kg[j], rtol=0, atol=1e-12 * np.abs(Kg).max())


def test_converges_to_exact_dse_under_refinement():
    # Keys cubic convolution is third order for values and second order for
    # first derivatives; the entry error of D-SKI against D-SE must fall at
    # about those rates as h -> 0 (the paper reports only "near 1e-5" with no
    # configuration, so the rate is the pin).
    X = _pts(12, 2, 8) * 0.6 + 0.2
    ell = [0.35, 0.3]
    exact = dse_matrix(X, ell, 1.0)
    n = 12
    errs_v, errs_g = [], []
    hs = []
    for m in [24, 48, 96, 192]:
        g = Grid(m=(m, m), lo=(-0.2, -0.2), hi=(1.2, 1.2))
        op = DSKI(X, g, ell, 1.0, 0.0, 0.0)
        E = np.abs(op.dense_kgrad() - exact)
        errs_v.append(E[:n, :n].max())
        errs_g.append(E[n:, n:].max() / np.abs(exact[n:, n:]).max())
        hs.append(g.h[0])
    rate_v = np.polyfit(np.log(hs), np.log(errs_v), 1)[0]
    rate_g = np.polyfit(np.log(hs), np.log(errs_g), 1)[0]
    assert rate_v > 2.6, (rate_v, errs_v)
    assert rate_g > 1.7, (rate_g, errs_g)
    assert errs_v[-1] < 1e-5


def test_abs_mvm_bounds_the_product():
    """abs_mvm is |B| K_UU |B|^T |v| + noise |v| (dense brute force) and
    dominates |K~ v| entrywise."""
    g = Grid(m=(9, 11), lo=(-0.3, -0.3), hi=(1.3, 1.3))
    X = _pts(30, 2, 8)
    op = DSKI(X, g, [0.3, 0.4], 1.2, 1e-3, 2e-3)
    v = np.random.default_rng(9).normal(size=op.N)
    Ba = np.abs(op.B.toarray())
    want = Ba @ kuu_dense(g, op.ell, op.sf) @ Ba.T @ np.abs(v) + op.noise * np.abs(v)
    assert np.allclose(op.abs_mvm(v), want, rtol=1e-13, atol=0)
    assert np.all(op.abs_mvm(v) >= np.abs(op.mvm(v)) * (1 - 1e-13))


def test_circulant_embedding_sizes():
    from oracle.dski import circulant_size
    assert [circulant_size(m) for m in (1, 2, 3, 4, 5, 256, 257, 1024, 1027)] == \
        [1, 4, 8, 8, 16, 512, 1024, 2048, 4096]


@pytest.mark.parametrize("m", [1, 2, 5, 17, 64])
def test_toeplitz_fft_apply_equals_dense(m):
    # the FFT product of a symmetric Toeplitz matrix equals the dense one
    from oracle.dski import toeplitz_fft_apply
    from scipy.linalg import toeplitz
    rng = np.random.default_rng(m)
    col = rng.normal(size=m)
    X = rng.normal(size=(m, 3))
    assert np.allclose(toeplitz_fft_apply(col, X), toeplitz(col) @ X, rtol=0, atol=1e-12 * m)


def test_kuu_apply_fft_equals_kronecker():
    from oracle.dski import kuu_apply_fft
    g = Grid(m=(9, 14, 6), lo=(0, -1, 0.5), hi=(1, 2, 1.5))
    ell = np.array([0.3, 0.9, 0.2])
    G = np.random.default_rng(8).normal(size=(g.size, 2))
    ref = kuu_apply(g, ell, 1.3, G)
    assert np.allclose(kuu_apply_fft(g, ell, 1.3, G), ref, rtol=0, atol=1e-13 * np.abs(ref).max() * 10)
