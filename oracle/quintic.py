"""Six-point quintic interpolation kernel (Sec. 3.1, D-SKI).

The paper interpolates with the quintic convolution kernel of Meijering,
Zuiderveld and Viergever (1999) and so has 6^d weights per row of W and dW.
That kernel is the member of the family of even, piecewise-quintic kernels
phi with knots at the integers and support (-3, 3) that

* interpolates: phi(0) = 1, phi(1) = phi(2) = 0;
* is three times continuously differentiable on the real line (at the knots
  1 and 2, and at 3 where it meets zero; at 0 evenness makes the odd
  derivatives vanish);

a one-parameter family, in which the single choice that reproduces
polynomials up to degree two (the highest order any member reaches) puts
3/64 as the leading coefficient of the outermost piece.  Written out in
s = |x| (the coefficients solve those conditions; the pins in
tests/test_oracle_quintic.py rederive them from the conditions alone):

    0 <= s <= 1:  -27/32 s^5 + 63/32 s^4 - 17/8 s^2 + 1
    1 <  s <= 2:   13/64 s^5 - 21/16 s^4 + 85/32 s^3 - 7/8 s^2 - 165/64 s + 61/32
    2 <  s <  3:    3/64 s^5 - 21/32 s^4 + 117/32 s^3 - 81/8 s^2 + 891/64 s - 243/32

Test infrastructure only (see ``oracle/__init__``).
"""
import numpy as np

# piece coefficients, lowest degree first, in s = |x|
PIECES = (
    (1.0, 0.0, -17 / 8, 0.0, 63 / 32, -27 / 32),
    (61 / 32, -165 / 64, -7 / 8, 85 / 32, -21 / 16, 13 / 64),
    (-243 / 32, 891 / 64, -81 / 8, 117 / 32, -21 / 32, 3 / 64),
)


def _piecewise(s, coef_of_piece):
    s = np.abs(np.asarray(s, dtype=np.float64))
    out = np.zeros_like(s)
    for k in range(3):
        if k == 0:
            sel = s <= 1.0
        elif k == 1:
            sel = (s > 1.0) & (s <= 2.0)
        else:
            sel = (s > 2.0) & (s < 3.0)
        out = np.where(sel, np.polynomial.polynomial.polyval(s, coef_of_piece(k)), out)
    return out


def omega5(s):
    """Quintic kernel value phi(s)."""
    return _piecewise(s, lambda k: PIECES[k])


def domega5(s):
    """Derivative d phi / d s (odd in s)."""
    s = np.asarray(s, dtype=np.float64)
    d = _piecewise(s, lambda k: np.polynomial.polynomial.polyder(PIECES[k]))
    return np.sign(s) * d


def stencil_1d(x, lo, hi, m):
    """Six-node stencil of one coordinate.

    t = (x - lo)/h, c = floor(t), nodes c-2 .. c+3 with weights phi(t - node)
    and derivative weights phi'(t - node)/h.  A point needs 2 <= c <= m-4 so
    that all six nodes exist.  Returns (nodes[6], w[6], dw[6]); raises
    ValueError out of grid.
    """
    h = (hi - lo) / (m - 1)
    t = (x - lo) / h
    c = int(np.floor(t))
    if c < 2 or c > m - 4:
        raise ValueError("point outside the interpolation grid")
    nodes = np.arange(c - 2, c + 4)
    s = t - nodes
    return nodes, omega5(s), domega5(s) / h
