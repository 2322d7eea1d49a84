"""Seeded synthetic stand-ins for the paper's workloads (Sec. 4).

The paper's datasets (Mount St. Helens LiDAR, the Stanford bunny, the test
function suite) are not available, so each workload is generated with the
shape, size and structure of the experiment it stands in for:

* ``sine2d``      n = 800 uniform points in [0,1]^2, f = sin(2 pi x1) cos(2 pi x2)
                  with its exact gradient; 32x32 grid.                (seed 1)
* ``terrain2d``   n = 100,000 uniform points in [0,1]^2, a 512-feature random
                  Fourier field (frequencies N(0, (8 pi)^2 I), amplitudes
                  N(0, 1/512), phases U[0, 2 pi)) with its gradient; 256x256
                  grid over [-0.05, 1.05]^2.  Terrain stand-in.      (seed 2)
* ``surface3d``   implicit surface of a bumpy sphere r = 1 + 0.15 Y, Y a real
                  spherical-harmonic series of degrees 1..6 normalised to
                  max|Y| = 1; 25,000 surface points (value 0) and 2,500 points
                  offset by +-0.05 along the normal (value +-0.05), gradients =
                  unit outward normals; 64^3 grid over [-1.4, 1.4]^3. Bunny
                  stand-in.                                          (seed 3)
* ``multi``       256 independent problems, d in {2, 3}, n log-uniform in
                  [200, 5000], 128-feature random Fourier targets, l ~ U[0.05, 0.3],
                  48^2 or 24^3 grids over [-0.1, 1.1]^d.       (seeds 4000+i)
* ``surface3d_big`` the surface3d generator at 50,000 + 5,000 points.  (seed 5)
* ``franke2d``    n = 2,000 uniform points in [0,1]^2 with Franke's test function
                  and its gradient (the preconditioning experiment of App. C);
                  96x96 grid over [-0.1, 1.1]^2.                     (seed 6)

Every vector is in block order [values (n); d/dx_1 (n); ...; d/dx_d (n)].
"""
import math

import numpy as np
from scipy.special import lpmv


def _problem(X, y, m, lo, hi, ell, sf, nv, ng, **extra):
    d = X.shape[1]
    out = dict(X=np.ascontiguousarray(X, np.float64), y=np.ascontiguousarray(y, np.float64),
               m=tuple(int(v) for v in m), lo=tuple(float(v) for v in lo),
               hi=tuple(float(v) for v in hi),
               ell=tuple(float(v) for v in (ell if np.ndim(ell) else [ell] * d)),
               sf=float(sf), noise_value=float(nv), noise_grad=float(ng))
    out.update(extra)
    return out


def rff_field(X, W, a, b):
    """f(x) = sum_j a_j cos(w_j.x + b_j) and grad f = -sum_j a_j w_j sin(.)."""
    arg = X @ W.T + b[None, :]
    f = np.cos(arg) @ a
    g = -(np.sin(arg) * a[None, :]) @ W
    return f, g


def sine2d(n=800, seed=1):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, (n, 2))
    s, c = np.sin(2 * np.pi * X[:, 0]), np.cos(2 * np.pi * X[:, 1])
    f = s * c
    fx = 2 * np.pi * np.cos(2 * np.pi * X[:, 0]) * c
    fy = -2 * np.pi * s * np.sin(2 * np.pi * X[:, 1])
    y = np.concatenate([f, fx, fy])
    return _problem(X, y, (32, 32), (-0.1, -0.1), (1.1, 1.1), 0.15, 1.0, 1e-4, 1e-4,
                    rank=20, rtol=1e-10, name="sine2d-n800-grid32")


def terrain2d(n=100_000, seed=2, features=512, grid=256):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, (n, 2))
    W = rng.normal(0.0, 8 * np.pi, (features, 2))
    a = rng.normal(0.0, math.sqrt(1.0 / features), features)
    b = rng.uniform(0.0, 2 * np.pi, features)
    f, g = rff_field(X, W, a, b)
    y = np.concatenate([f, g[:, 0], g[:, 1]])
    return _problem(X, y, (grid, grid), (-0.05, -0.05), (1.05, 1.05), 0.05, 1.0, 1e-3, 1e-3,
                    rank=100, rtol=1e-8, name=f"terrain2d-n{n}-grid{grid}")


def _real_sh(l, m, theta, phi):
    """Real spherical harmonic (unnormalised Legendre form; normalisation is
    irrelevant because the series is rescaled to max|Y| = 1)."""
    P = lpmv(abs(m), l, np.cos(theta))
    if m > 0:
        return P * np.cos(m * phi)
    if m < 0:
        return P * np.sin(-m * phi)
    return P


class BumpySphere:
    def __init__(self, rng, lmax=6, amp=0.15):
        self.terms = [(l, m, rng.normal()) for l in range(1, lmax + 1) for m in range(-l, l + 1)]
        self.amp = amp
        check = rng.normal(size=(100_000, 3))
        th, ph = self._angles(check)
        self.scale = 1.0 / np.abs(self._Y(th, ph)).max()

    @staticmethod
    def _angles(P):
        r = np.linalg.norm(P, axis=1)
        return np.arccos(np.clip(P[:, 2] / r, -1, 1)), np.arctan2(P[:, 1], P[:, 0])

    def _Y(self, th, ph):
        return sum(c * _real_sh(l, m, th, ph) for l, m, c in self.terms)

    def radius(self, P):
        th, ph = self._angles(P)
        return 1.0 + self.amp * self.scale * self._Y(th, ph)

    def F(self, P):
        return np.linalg.norm(P, axis=1) - self.radius(P)

    def normal(self, P, h=1e-6):
        G = np.empty_like(P)
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            G[:, k] = (self.F(P + e) - self.F(P - e)) / (2 * h)
        return G / np.linalg.norm(G, axis=1)[:, None]


def surface3d(n_surface=25_000, n_offset=2_500, seed=3, grid=64, offset=0.05):
    rng = np.random.default_rng(seed)
    S = BumpySphere(rng)
    dirs = rng.normal(size=(n_surface, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    Xs = dirs * S.radius(dirs)[:, None]
    Ns = S.normal(Xs)
    dirs2 = rng.normal(size=(n_offset, 3))
    dirs2 /= np.linalg.norm(dirs2, axis=1)[:, None]
    base = dirs2 * S.radius(dirs2)[:, None]
    Nb = S.normal(base)
    sign = rng.choice([-1.0, 1.0], n_offset)
    Xo = base + offset * sign[:, None] * Nb
    X = np.vstack([Xs, Xo])
    vals = np.concatenate([np.zeros(n_surface), offset * sign])
    G = np.vstack([Ns, Nb])
    y = np.concatenate([vals, G[:, 0], G[:, 1], G[:, 2]])
    return _problem(X, y, (grid,) * 3, (-1.4,) * 3, (1.4,) * 3, 0.2, 1.0, 1e-4, 1e-4,
                    rank=100, rtol=1e-8, probes=31, depth=30,
                    name=f"surface3d-n{n_surface + n_offset}-grid{grid}")


def surface3d_big(seed=5):
    p = surface3d(50_000, 5_000, seed=seed)
    p.update(probes=16, name="surface3d-n55000-grid64")
    return p


def multi_instance(i, seed_base=4000):
    rng = np.random.default_rng(seed_base + i)
    d = int(rng.choice([2, 3]))
    n = int(round(math.exp(rng.uniform(math.log(200), math.log(5000)))))
    ell = rng.uniform(0.05, 0.3)
    X = rng.uniform(0.0, 1.0, (n, d))
    W = rng.normal(0.0, 1.0 / ell, (128, d))
    a = rng.normal(0.0, math.sqrt(1.0 / 128), 128)
    b = rng.uniform(0.0, 2 * np.pi, 128)
    f, g = rff_field(X, W, a, b)
    y = np.concatenate([f] + [g[:, k] for k in range(d)])
    m = 48 if d == 2 else 24
    return _problem(X, y, (m,) * d, (-0.1,) * d, (1.1,) * d, ell, 1.0, 1e-3, 1e-3,
                    rank=32, rtol=1e-6, name=f"multi-{i}")


def franke(X):
    """Franke's bivariate test function (Franke 1979) and its gradient."""
    x, y = 9 * X[:, 0], 9 * X[:, 1]
    t1 = 0.75 * np.exp(-((x - 2) ** 2 + (y - 2) ** 2) / 4)
    t2 = 0.75 * np.exp(-((x + 1) ** 2) / 49 - (y + 1) / 10)
    t3 = 0.5 * np.exp(-((x - 7) ** 2 + (y - 3) ** 2) / 4)
    t4 = -0.2 * np.exp(-((x - 4) ** 2) - (y - 7) ** 2)
    f = t1 + t2 + t3 + t4
    fx = 9 * (t1 * (-(x - 2) / 2) + t2 * (-2 * (x + 1) / 49) + t3 * (-(x - 7) / 2)
              + t4 * (-2 * (x - 4)))
    fy = 9 * (t1 * (-(y - 2) / 2) + t2 * (-1 / 10) + t3 * (-(y - 3) / 2) + t4 * (-2 * (y - 7)))
    return f, fx, fy


def franke2d(n=2000, seed=6, ell=0.1, noise=1e-2, grid=96):
    """The preconditioning experiment's 2-D workload (App. C): n points
    uniform in [0,1]^2 with Franke's function and its gradient, SE output
    scale 1, one length scale and noise; grid over [-0.1, 1.1]^2."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, (n, 2))
    f, fx, fy = franke(X)
    return _problem(X, np.concatenate([f, fx, fy]), (grid, grid), (-0.1, -0.1), (1.1, 1.1),
                    ell, 1.0, noise, noise, rank=100, rtol=1e-4, name=f"franke2d-n{n}")


def subsample(p, n, seed=0):
    """Seeded subsample of a problem's points (values and gradients kept together)."""
    X = p["X"]
    N0, d = X.shape
    idx = np.sort(np.random.default_rng(seed).choice(N0, n, replace=False))
    y = p["y"].reshape(d + 1, N0)[:, idx].ravel()
    q = dict(p)
    q.update(X=X[idx].copy(), y=y)
    return q


def small2d(n, m=16, seed=0, ell=0.2, nv=1e-3, ng=1e-3, lo=-0.2, hi=1.2):
    """Small random 2-D problem for parity tests."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, (n, 2))
    y = rng.normal(size=3 * n)
    return _problem(X, y, (m, m + 3), (lo, lo), (hi, hi), (ell, ell * 1.3), 1.1, nv, ng,
                    name=f"small2d-n{n}")


def small3d(n, m=12, seed=0, ell=0.3, nv=1e-3, ng=2e-3):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, (n, 3))
    y = rng.normal(size=4 * n)
    return _problem(X, y, (m, m + 1, m + 2), (-0.3,) * 3, (1.3,) * 3, (ell, ell * 0.8, ell * 1.2),
                    0.9, nv, ng, name=f"small3d-n{n}")
