"""Pins of the six-point quintic kernel (Sec. 3.1, Meijering et al. 1999)
and of the quintic D-SKI operator.

The kernel is fixed by its defining conditions, so the first pin rederives
its eighteen coefficients from them alone (a linear system written here, not
the oracle's table): evenness at 0 (phi' = phi''' = 0), interpolation at the
knots, C^3 continuity at 1 and 2, vanishing with three derivatives at 3, and
reproduction of linear functions (one equation at f = 0.3 fixes the one free
parameter).  The rest check the properties that follow: partition of unity,
exact quadratics and their derivatives, cubics not exact, the 6^d stencil
bounds, and the accuracy gain over Keys' cubic kernel that the paper gives
as its reason for the quintic scheme."""
import numpy as np
import pytest

from oracle import keys
from oracle.dse import dse_matrix
from oracle.dski import DSKI, Grid, interp_matrix
from oracle.quintic import PIECES, domega5, omega5, stencil_1d


def _dpoly(j, x, r):
    """r-th derivative of x^j at x."""
    if r > j:
        return 0.0
    c = 1.0
    for t in range(r):
        c *= (j - t)
    return c * x ** (j - r)


def _row(piece, x, r):
    row = np.zeros(18)
    for j in range(6):
        row[6 * piece + j] = _dpoly(j, x, r)
    return row


def test_coefficients_follow_from_the_defining_conditions():
    A, b = [], []
    A += [_row(0, 0.0, 1), _row(0, 0.0, 3)]
    b += [0.0, 0.0]
    for piece, x, v in [(0, 0.0, 1.0), (0, 1.0, 0.0), (1, 1.0, 0.0), (1, 2.0, 0.0),
                        (2, 2.0, 0.0), (2, 3.0, 0.0)]:
        A.append(_row(piece, x, 0))
        b.append(v)
    for r in (1, 2, 3):
        A.append(_row(0, 1.0, r) - _row(1, 1.0, r))
        A.append(_row(1, 2.0, r) - _row(2, 2.0, r))
        A.append(_row(2, 3.0, r))
        b += [0.0, 0.0, 0.0]
    # sum_k phi(f - k) k = f at f = 0.3, nodes k = -2..3 at distances |f - k|
    f = 0.3
    row = np.zeros(18)
    for k in range(-2, 4):
        dist = abs(f - k)
        piece = min(int(dist), 2)
        row += k * _row(piece, dist, 0)
    A.append(row)
    b.append(f)
    coef = np.linalg.solve(np.array(A), np.array(b))
    assert np.allclose(coef.reshape(3, 6), np.array(PIECES), rtol=1e-11, atol=1e-11)
    assert abs(PIECES[2][5] - 3 / 64) < 1e-16


def test_special_values_and_symmetry():
    s = np.array([0.0, 1.0, 2.0, 3.0, 3.5, 0.5, 1.5, 2.5])
    want = [1, 0, 0, 0, 0, 1 - 17 / 32 + 63 / 512 - 27 / 1024,
            None, 3 / 64 * 0.5 * 0.5**4]
    got = omega5(s)
    for g, w in zip(got, want):
        if w is not None:
            assert abs(g - w) < 1e-14
    x = np.linspace(-3.2, 3.2, 129)
    assert np.allclose(omega5(x), omega5(-x), atol=1e-15)
    assert np.allclose(domega5(x), -domega5(-x), atol=1e-15)


def test_derivative_matches_finite_differences_and_is_continuous():
    s = np.linspace(-2.9, 2.9, 117) + 1e-3
    h = 1e-6
    fd = (omega5(s + h) - omega5(s - h)) / (2 * h)
    assert np.allclose(domega5(s), fd, atol=1e-8)
    for k in (1.0, 2.0, 3.0):
        e = 1e-9
        assert abs(omega5(k - e) - omega5(k + e)) < 1e-8
        assert abs(domega5(k - e) - domega5(k + e)) < 1e-7


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_reproduces_quadratics_and_their_derivatives(deg):
    rng = np.random.default_rng(10 + deg)
    lo, hi, m = -0.3, 1.4, 37
    h = (hi - lo) / (m - 1)
    p = np.polynomial.Polynomial(rng.normal(size=deg + 1))
    for _ in range(40):
        x = rng.uniform(lo + 2.0 * h, hi - 2.0 * h - 1e-9)
        nodes, w, dw = stencil_1d(x, lo, hi, m)
        u = lo + nodes * h
        assert abs(w @ p(u) - p(x)) < 1e-12
        assert abs(dw @ p(u) - p.deriv()(x)) < 1e-9


def test_cubics_are_not_reproduced():
    nodes, w, _ = stencil_1d(0.537, 0.0, 1.0, 11)
    u = nodes * 0.1
    assert abs(w @ u**3 - 0.537**3) > 1e-6


def test_stencil_bounds_and_grid_line():
    nodes, w, _ = stencil_1d(0.375, 0.0, 1.0, 9)     # h = 1/8, t = 3 exactly
    assert list(nodes) == [1, 2, 3, 4, 5, 6]
    assert np.allclose(w, [0, 0, 1, 0, 0, 0], atol=1e-15)
    with pytest.raises(ValueError):
        stencil_1d(0.15, 0.0, 1.0, 11)   # c = 1 lacks node c-2
    nodes, _, _ = stencil_1d(0.25, 0.0, 1.0, 11)    # c = 2: first valid cell
    assert list(nodes) == [0, 1, 2, 3, 4, 5]
    nodes, _, _ = stencil_1d(0.75, 0.0, 1.0, 11)    # c = 7 = m-4: last valid cell
    assert list(nodes) == [5, 6, 7, 8, 9, 10]
    with pytest.raises(ValueError):
        stencil_1d(0.85, 0.0, 1.0, 11)   # c = 8 lacks node c+3


def test_more_accurate_than_cubic_on_smooth_functions():
    # the paper's reason for the quintic scheme: smaller interpolation error
    f = lambda x: np.sin(5.0 * x) + 0.3 * np.cos(11.0 * x)
    df = lambda x: 5.0 * np.cos(5.0 * x) - 3.3 * np.sin(11.0 * x)
    lo, hi, m = -0.3, 1.3, 33
    h = (hi - lo) / (m - 1)
    xs = np.linspace(0.0, 1.0, 401)
    err = {}
    for name, st in (("cubic", keys.stencil_1d), ("quintic", stencil_1d)):
        e0 = e1 = 0.0
        for x in xs:
            nodes, w, dw = st(x, lo, hi, m)
            u = lo + nodes * h
            e0 = max(e0, abs(w @ f(u) - f(x)))
            e1 = max(e1, abs(dw @ f(u) - df(x)))
        err[name] = (e0, e1)
    # both kernels reproduce quadratics (errors O(h^3), O(h^2) for the
    # derivative); the quintic's constants are smaller: ~0.74x and ~0.46x
    # on this grid (~0.65x and ~0.44x as h -> 0)
    assert err["quintic"][0] < 0.8 * err["cubic"][0]
    assert err["quintic"][1] < 0.6 * err["cubic"][1]


@pytest.mark.parametrize("d", [1, 2, 3])
def test_quintic_rows(d):
    g = Grid(m=(12,) * d, lo=(-0.3,) * d, hi=(1.3,) * d, interp="quintic")
    X = np.random.default_rng(d).uniform(0, 1, (30, d))
    B = interp_matrix(X, g).toarray()
    n = X.shape[0]
    assert np.allclose(B[:n].sum(1), 1.0, atol=1e-13)
    assert np.allclose(B[n:].sum(1), 0.0, atol=1e-9)
    assert np.all((B[:n] != 0).sum(1) <= 6**d)
    assert np.any((B[:n] != 0).sum(1) > 4**d)


def test_quintic_dski_closer_to_exact_kernel():
    # K~ with the quintic stencil approximates the exact derivative SE
    # kernel matrix (Sec. 2) more closely than the cubic one on the same grid
    rng = np.random.default_rng(7)
    X = rng.uniform(0, 1, (40, 2))
    ell, sf = [0.25, 0.3], 1.0
    K = dse_matrix(X, np.array(ell), sf)
    errs = {}
    for interp in ("cubic", "quintic"):
        g = Grid(m=(20, 20), lo=(-0.35, -0.35), hi=(1.35, 1.35), interp=interp)
        op = DSKI(X, g, ell, sf, 1e-3, 1e-3)
        errs[interp] = np.abs(op.dense_kgrad() - K).max() / np.abs(K).max()
    assert errs["quintic"] < 0.7 * errs["cubic"], errs   # ~0.59x here


def test_quintic_diag_and_rows_match_dense():
    g = Grid(m=(13, 11), lo=(-0.4, -0.45), hi=(1.3, 1.4), interp="quintic")
    X = np.random.default_rng(3).uniform(0, 1, (25, 2))
    op = DSKI(X, g, [0.3, 0.35], 1.2, 1e-3, 1e-3)
    Kg = op.dense_kgrad()
    assert np.allclose(op.kgrad_diag(), np.diag(Kg), rtol=1e-12, atol=0)
    for j in (0, 27, 61):
        assert np.allclose(op.kgrad_row(j), Kg[j], rtol=0, atol=1e-12 * np.abs(Kg).max())
