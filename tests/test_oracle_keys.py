"""Pins of the Keys cubic-convolution kernel (Sec. 3.1) against closed forms
and the polynomial-reproduction property of Keys' a = -1/2 kernel."""
import numpy as np
import pytest

from oracle.keys import omega, domega, stencil_1d


def test_special_values():
    # Keys' kernel interpolates (1 at 0, 0 at the other integers) and
    # takes 9/16 at 1/2 and -1/16 at 3/2 for a = -1/2.
    s = np.array([0.0, 1.0, -1.0, 2.0, -2.0, 0.5, -0.5, 1.5, -1.5, 2.5])
    want = np.array([1, 0, 0, 0, 0, 9 / 16, 9 / 16, -1 / 16, -1 / 16, 0])
    assert np.allclose(omega(s), want, atol=1e-15)


def test_derivative_matches_finite_differences():
    s = np.linspace(-2.4, 2.4, 97) + 1e-3
    h = 1e-6
    fd = (omega(s + h) - omega(s - h)) / (2 * h)
    assert np.allclose(domega(s), fd, atol=1e-8)


def test_c1_continuity_at_knots():
    for k in [1.0, 2.0]:
        e = 1e-9
        assert abs(omega(k - e) - omega(k + e)) < 1e-8
        assert abs(domega(k - e) - domega(k + e)) < 1e-7


def test_partition_of_unity_and_zero_derivative_sum():
    rng = np.random.default_rng(0)
    for _ in range(50):
        x = rng.uniform(0.3, 0.7)
        nodes, w, dw = stencil_1d(x, 0.0, 1.0, 21)
        assert abs(w.sum() - 1.0) < 1e-14
        assert abs(dw.sum()) < 1e-11


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_reproduces_quadratics_and_their_derivatives(deg):
    rng = np.random.default_rng(deg)
    lo, hi, m = -0.3, 1.4, 37
    h = (hi - lo) / (m - 1)
    c = rng.normal(size=deg + 1)
    p = np.polynomial.Polynomial(c)
    for _ in range(40):
        x = rng.uniform(lo + 1.5 * h, hi - 2.5 * h)
        nodes, w, dw = stencil_1d(x, lo, hi, m)
        u = lo + nodes * h
        assert abs(w @ p(u) - p(x)) < 1e-12
        assert abs(dw @ p(u) - p.deriv()(x)) < 1e-9


def test_cubics_are_not_reproduced():
    # negative control: the a = -1/2 kernel is exact to degree 2 only
    lo, hi, m = 0.0, 1.0, 11
    h = 0.1
    x = 0.537
    nodes, w, _ = stencil_1d(x, lo, hi, m)
    u = lo + nodes * h
    assert abs(w @ u**3 - x**3) > 1e-6


def test_grid_line_and_out_of_grid():
    nodes, w, _ = stencil_1d(0.375, 0.0, 1.0, 9)     # h = 1/8 exactly, t = 3
    assert list(nodes) == [2, 3, 4, 5]
    assert np.allclose(w, [0, 1, 0, 0], atol=1e-15)
    with pytest.raises(ValueError):
        stencil_1d(0.05, 0.0, 1.0, 11)   # c = 0 lacks node c-1
    nodes, _, _ = stencil_1d(0.85, 0.0, 1.0, 11)   # c = 8 = m-3: last valid cell
    assert list(nodes) == [7, 8, 9, 10]
    with pytest.raises(ValueError):
        stencil_1d(0.95, 0.0, 1.0, 11)   # c = 9 lacks node c+2
