"""Keys cubic-convolution interpolation kernel (Sec. 3.1, D-SKI).

The paper differentiates the interpolation scheme rather than the kernel:
k(x, x') ~ sum_i w_i(x) k(u_i, x') and grad k ~ sum_i grad w_i(x) k(u_i, x').
It names cubic convolution (Keys, 1981) as one admissible scheme; the build
uses it with Keys' parameter a = -1/2, which gives a 4-point stencil per
dimension and reproduces polynomials up to degree two.

Test infrastructure only (see ``oracle/__init__``).
"""
import numpy as np

KEYS_A = -0.5


def omega(s, a=KEYS_A):
    """Keys kernel value.  |s| <= 1: (a+2)|s|^3 - (a+3)|s|^2 + 1;
    1 < |s| < 2: a|s|^3 - 5a|s|^2 + 8a|s| - 4a; 0 otherwise."""
    s = np.abs(np.asarray(s, dtype=np.float64))
    inner = (a + 2.0) * s**3 - (a + 3.0) * s**2 + 1.0
    outer = a * s**3 - 5.0 * a * s**2 + 8.0 * a * s - 4.0 * a
    return np.where(s <= 1.0, inner, np.where(s < 2.0, outer, 0.0))


def domega(s, a=KEYS_A):
    """Derivative d omega / d s of the Keys kernel (odd in s)."""
    s = np.asarray(s, dtype=np.float64)
    t = np.abs(s)
    sg = np.sign(s)
    inner = 3.0 * (a + 2.0) * t**2 - 2.0 * (a + 3.0) * t
    outer = 3.0 * a * t**2 - 10.0 * a * t + 8.0 * a
    return sg * np.where(t <= 1.0, inner, np.where(t < 2.0, outer, 0.0))


def grid_spacing(lo, hi, m):
    """Regular grid u_a = lo + a*h, a = 0..m-1, both end points included."""
    return (hi - lo) / (m - 1)


def stencil_1d(x, lo, hi, m):
    """Four-node stencil of one coordinate.

    t = (x - lo)/h, c = floor(t), nodes c-1, c, c+1, c+2 with weights
    omega(t - node) and derivative weights omega'(t - node)/h (chain rule
    for d/dx).  A point needs 1 <= c <= m-3 so that all four nodes exist.

    Returns (nodes[4] int, w[4], dw[4]); raises ValueError out of grid.
    """
    h = grid_spacing(lo, hi, m)
    t = (x - lo) / h
    c = int(np.floor(t))
    if c < 1 or c > m - 3:
        raise ValueError("point outside the interpolation grid")
    nodes = np.arange(c - 1, c + 3)
    s = t - nodes
    return nodes, omega(s), domega(s) / h
