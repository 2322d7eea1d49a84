"""Pins of the marginal-likelihood oracle (Eq. 1): the value against SciPy's
multivariate normal density, the exact gradient against central finite
differences, and the Hutchinson gradient against the exact one with scaled
basis probes (an exact trace)."""
import numpy as np
import pytest
import scipy.stats as st

from oracle.dski import DSKI, Grid
from oracle.mll import mll_dense, mll_grad_dense, mll_grad_hutchinson, mll_grad_hutchinson_z
from oracle.solve import pivoted_cholesky, QRPreconditioner


def _make(theta, X, grid, rho):
    d = X.shape[1]
    ell = np.exp(theta[:d])
    sf = np.exp(theta[d])
    s2 = np.exp(2 * theta[d + 1])
    return DSKI(X, grid, ell, sf, s2, rho * s2)


def _setup(n=10, d=2, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (n, d))
    grid = Grid(m=(10,) * d, lo=(-0.3,) * d, hi=(1.3,) * d)
    theta = np.array([np.log(0.35), np.log(0.3), np.log(1.2), np.log(0.1)])[: d + 2] if d == 2 else \
        np.array([np.log(0.35), np.log(0.4), np.log(0.3), np.log(1.2), np.log(0.1)])
    y = rng.normal(size=n * (d + 1))
    return X, grid, theta, y


def test_mll_value_is_gaussian_log_density():
    X, grid, theta, y = _setup()
    op = _make(theta, X, grid, 2.0)
    want = st.multivariate_normal(mean=np.zeros(op.N), cov=op.dense()).logpdf(y)
    assert abs(mll_dense(op, y) - want) < 1e-9 * abs(want)


def test_gradient_matches_central_differences():
    for d in (2, 3):
        X, grid, theta, y = _setup(n=8, d=d, seed=d)
        g = mll_grad_dense(_make(theta, X, grid, 2.0), y)
        h = 1e-4
        for i in range(d + 2):
            e = np.zeros_like(theta)
            e[i] = h
            fd = (mll_dense(_make(theta + e, X, grid, 2.0), y)
                  - mll_dense(_make(theta - e, X, grid, 2.0), y)) / (2 * h)
            assert abs(g[i] - fd) < 1e-6 * max(1.0, abs(fd)), (d, i, g[i], fd)


def test_hutchinson_with_basis_probes_is_exact():
    X, grid, theta, y = _setup(n=6, seed=4)
    op = _make(theta, X, grid, 2.0)
    L, _, _ = pivoted_cholesky(op.kgrad_diag(), op.kgrad_row, 5)
    Pc = QRPreconditioner(L, op.noise)
    W = np.sqrt(op.N) * np.eye(op.N)
    _, _, g = mll_grad_hutchinson(op, y, Pc, W, rtol=1e-14)
    ge = mll_grad_dense(op, y)
    assert np.allclose(g, ge, rtol=1e-7, atol=1e-7)


def test_hutchinson_with_factor_basis_probes_is_exact():
    X, grid, theta, y = _setup(n=6, seed=5)
    op = _make(theta, X, grid, 2.0)
    L, _, _ = pivoted_cholesky(op.kgrad_diag(), op.kgrad_row, 4)
    Pc = QRPreconditioner(L, op.noise)
    P = op.N + 4
    Z = np.sqrt(P) * Pc.factor_apply(np.eye(P))
    _, _, g = mll_grad_hutchinson_z(op, y, Pc, Z, rtol=1e-14)
    assert np.allclose(g, mll_grad_dense(op, y), rtol=1e-7, atol=1e-7)


@pytest.mark.parametrize("d,m,interp", [(2, (9, 11), "cubic"), (3, (7, 8, 9), "cubic"),
                                        (2, (11, 13), "quintic"), (3, (9, 10, 11), "quintic")])
def test_factored_dense_matrices_equal_the_kronecker_ones(d, m, interp):
    # the per-dimension (Hadamard) form of B K_UU B^T and of every dK~/dtheta
    # equals the one through the dense K_UU
    from oracle.dski import dense_kgrad_factored, kfactor
    from oracle.mll import dtheta_dense_factored, dtheta_mvm
    X = np.random.default_rng(1).uniform(0, 1, (15, d))
    g = Grid(m, (-0.6,) * d, (1.6,) * d, interp)
    op = DSKI(X, g, [0.3, 0.4, 0.5][:d], 1.3, 1e-3, 2e-3)
    A = op.dense_kgrad()
    B = dense_kgrad_factored(X, g, [kfactor(g, k, op.ell[k]) for k in range(d)], op.sf)
    assert np.allclose(B, A, rtol=0, atol=1e-14 * np.abs(A).max())
    for i in range(d + 2):
        Di = dtheta_mvm(op, i, np.eye(op.N))
        assert np.allclose(dtheta_dense_factored(op, i), Di, rtol=0, atol=1e-13 * np.abs(Di).max())


def test_surface_subsample_gradient_matches_central_differences():
    # the 3-D bumpy-surface generator at 55,000 points, seeded n = 1,000
    # subsample, theta = (log 0.2 x 3, log 1, log 1e-2): the exact gradient of
    # Eq. 1 against central differences of the exact L with step 1e-4
    from synth import workloads as W
    from oracle.mll import mll_dense, mll_grad_dense
    p = W.subsample(W.surface3d_big(), 1000, seed=0)

    def op_at(th):
        s2 = np.exp(2 * th[4])
        return DSKI(p["X"], Grid(p["m"], p["lo"], p["hi"]), np.exp(th[:3]), np.exp(th[3]), s2, s2)

    th = np.array([np.log(0.2)] * 3 + [0.0, 0.5 * np.log(1e-4)])
    g = mll_grad_dense(op_at(th), p["y"], factored=True)
    h = 1e-4
    for i in range(5):
        e = np.zeros(5)
        e[i] = h
        fd = (mll_dense(op_at(th + e), p["y"], factored=True)
              - mll_dense(op_at(th - e), p["y"], factored=True)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * abs(g[i]), (i, fd, g[i])


def test_direct_hutchinson_equals_pcg_hutchinson_with_same_probes():
    """The dense-Cholesky form of the same-probe estimator equals the PCG
    form (solves to 1e-13) on the same probes, with K~ formed either way."""
    from oracle.mll import mll_grad_hutchinson_direct
    from oracle.probes import preconditioned_probes
    X, grid, theta, y = _setup(n=12, seed=6)
    op = _make(theta, X, grid, 2.0)
    L, _, _ = pivoted_cholesky(op.kgrad_diag(), op.kgrad_row, 6)
    Pc = QRPreconditioner(L, op.noise)
    Z = preconditioned_probes(17, Pc, 5)
    fit, tr, g = mll_grad_hutchinson_z(op, y, Pc, Z, rtol=1e-13)
    for factored in (False, True):
        fit2, tr2, g2 = mll_grad_hutchinson_direct(op, y, Pc, Z, factored=factored)
        assert np.allclose(fit2, fit, rtol=1e-9, atol=0)
        assert np.allclose(tr2, tr, rtol=1e-9, atol=1e-12)
        assert np.allclose(g2, g, rtol=1e-9, atol=1e-12)
