"""D-SKI (Sec. 3.1): K^grad ~ [W; dW] K_UU [W; dW]^T, plus the noise diagonal.

* U is a regular grid with m_k nodes per dimension from lo_k to hi_k (both
  ends included), flattened in C order (last dimension fastest).
* K_UU = s_f^2 K_1 (x) ... (x) K_d with K_k[a, b] = exp(-(u_a - u_b)^2 / 2 l_k^2):
  the SE kernel of App. A is a product over dimensions, so on a tensor grid
  it is a Kronecker product.
* W holds tensor-product interpolation weights w_i(u) = prod_k phi(t_ik - u_k)
  with phi Keys' cubic kernel (4 nodes per dimension) or the paper's
  six-point quintic kernel (6 nodes per dimension), as the grid's ``interp``
  says; dW_p differentiates them in dimension p only (phi'/h_p there).
* K~ = B K_UU B^T + diag(noise) with B = [W; dW_1; ...; dW_d] (N x m,
  N = n(d+1)), noise sigma_v^2 on value rows and sigma_g^2 on gradient rows.

Test infrastructure only (see ``oracle/__init__``).
"""
from dataclasses import dataclass
import itertools

import numpy as np
import scipy.sparse as sp

from .keys import omega, domega
from .quintic import omega5, domega5


@dataclass(frozen=True)
class Grid:
    """Regular grid plus the interpolation scheme on it ("cubic" or "quintic")."""
    m: tuple
    lo: tuple
    hi: tuple
    interp: str = "cubic"

    @property
    def stencil(self):
        """(nodes per dimension S, offset of the first node below floor(t))."""
        return (6, 2) if self.interp == "quintic" else (4, 1)

    @property
    def d(self):
        return len(self.m)

    @property
    def h(self):
        return tuple((b - a) / (mk - 1) for a, b, mk in zip(self.lo, self.hi, self.m))

    @property
    def size(self):
        return int(np.prod(self.m))

    def nodes(self, k):
        return self.lo[k] + np.arange(self.m[k]) * self.h[k]


def kfactor(grid, k, ell):
    """K_k[a, b] = exp(-(u_a - u_b)^2 / (2 l^2)) on dimension k of the grid."""
    u = grid.nodes(k)
    diff = u[:, None] - u[None, :]
    return np.exp(-0.5 * diff**2 / ell**2)


def kfactor_dlogell(grid, k, ell):
    """d K_k / d log l = K_k * (u_a - u_b)^2 / l^2."""
    u = grid.nodes(k)
    diff = u[:, None] - u[None, :]
    return np.exp(-0.5 * diff**2 / ell**2) * diff**2 / ell**2


def kuu_dense(grid, lengthscale, outputscale):
    """Dense K_UU = s_f^2 kron(K_1, ..., K_d) (small grids only)."""
    out = np.array([[1.0]])
    for k in range(grid.d):
        out = np.kron(out, kfactor(grid, k, lengthscale[k]))
    return outputscale**2 * out


def kron_apply(factors, G):
    """(A_1 (x) ... (x) A_d) G for G of shape (prod m_k, s), one mode at a time."""
    m = [A.shape[0] for A in factors]
    s = G.shape[1]
    T = G.reshape(*m, s)
    for k, A in enumerate(factors):
        T = np.moveaxis(np.tensordot(A, T, axes=([1], [k])), 0, k)
    return T.reshape(-1, s)


def kuu_apply(grid, lengthscale, outputscale, G):
    """K_UU G through the Kronecker factors (no dense K_UU)."""
    facs = [kfactor(grid, k, lengthscale[k]) for k in range(grid.d)]
    return outputscale**2 * kron_apply(facs, G)


def circulant_size(m):
    """Smallest power of two L >= 2 m - 1: an m x m Toeplitz matrix embeds in
    the leading block of an L x L circulant."""
    L = 1
    while L < 2 * m - 1:
        L *= 2
    return L


def toeplitz_fft_apply(col, X):
    """T X for the symmetric Toeplitz T with first column col (m entries), by
    circulant embedding and the FFT (Sec. 3.1: on a regular grid the SE
    factors are Toeplitz, and FFTs give O(m log m) products with K_UU).
    The circulant's first column is [col, 0 ..., col reversed without col[0]];
    its eigenvalues are the DFT of that column, so T x is the first m entries
    of IFFT(DFT(c) * FFT(x zero-padded to L))."""
    col = np.asarray(col, np.float64)
    X = np.asarray(X, np.float64)
    m = col.shape[0]
    L = circulant_size(m)
    c = np.zeros(L)
    c[:m] = col
    if m > 1:
        c[L - m + 1:] = col[1:][::-1]
    Xp = np.zeros((L,) + X.shape[1:])
    Xp[:m] = X
    lam = np.fft.fft(c)
    spec = np.fft.fft(Xp, axis=0) * lam.reshape((L,) + (1,) * (X.ndim - 1))
    return np.fft.ifft(spec, axis=0).real[:m]


def kuu_apply_fft(grid, lengthscale, outputscale, G):
    """K_UU G with each Kronecker factor applied by its circulant embedding
    (the same product as kuu_apply, in O(M sum_k log m_k))."""
    m = list(grid.m)
    s = G.shape[1]
    T = np.asarray(G, np.float64).reshape(*m, s)
    for k in range(grid.d):
        col = kfactor(grid, k, lengthscale[k])[:, 0]
        T = np.moveaxis(toeplitz_fft_apply(col, np.moveaxis(T, k, 0)), 0, k)
    return outputscale**2 * T.reshape(-1, s)


def stencils(X, grid):
    """Per point and dimension: first node c_k - lead, weights and derivative
    weights of the S stencil nodes (t = (x - lo)/h, c = floor(t); S = 4,
    lead = 1 for the cubic kernel, S = 6, lead = 2 for the quintic)."""
    X = np.asarray(X, np.float64)
    n, d = X.shape
    S, lead = grid.stencil
    phi, dphi = (omega5, domega5) if grid.interp == "quintic" else (omega, domega)
    first = np.empty((n, d), np.int64)
    w = np.empty((n, d, S))
    dw = np.empty((n, d, S))
    for k in range(d):
        h = grid.h[k]
        t = (X[:, k] - grid.lo[k]) / h
        c = np.floor(t).astype(np.int64)
        if np.any(c < lead) or np.any(c > grid.m[k] - S + lead):
            raise ValueError("point outside the interpolation grid")
        first[:, k] = c - lead
        s = t[:, None] - (c[:, None] - lead + np.arange(S)[None, :])
        w[:, k, :] = phi(s)
        dw[:, k, :] = dphi(s) / h
    return first, w, dw


def interp_matrix(X, grid):
    """Explicit sparse B = [W; dW_1; ...; dW_d] (N x m CSR)."""
    first, w, dw = stencils(X, grid)
    n, d = first.shape
    strides = [int(np.prod(grid.m[k + 1:])) for k in range(d)]
    rows, cols, vals = [], [], []
    pts = np.arange(n)
    for offs in itertools.product(range(w.shape[2]), repeat=d):
        col = np.zeros(n, np.int64)
        for k in range(d):
            col += (first[:, k] + offs[k]) * strides[k]
        wv = np.ones(n)
        for k in range(d):
            wv = wv * w[:, k, offs[k]]
        rows.append(pts)
        cols.append(col)
        vals.append(wv)
        for p in range(d):
            gv = np.ones(n)
            for k in range(d):
                gv = gv * (dw[:, k, offs[k]] if k == p else w[:, k, offs[k]])
            rows.append((p + 1) * n + pts)
            cols.append(col)
            vals.append(gv)
    B = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n * (d + 1), grid.size))
    return B.tocsr()


def interp_matrix_1d(X, grid, k):
    """Per-dimension interpolation matrices of dimension k: W_k and dW_k
    (n x m_k, the S weights and derivative weights of each point's stencil
    in that dimension)."""
    first, w, dw = stencils(X, grid)
    n, S = w.shape[0], w.shape[2]
    Wk = np.zeros((n, grid.m[k]))
    Dk = np.zeros((n, grid.m[k]))
    rows = np.repeat(np.arange(n), S)
    cols = (first[:, k][:, None] + np.arange(S)[None, :]).ravel()
    np.add.at(Wk, (rows, cols), w[:, k, :].ravel())
    np.add.at(Dk, (rows, cols), dw[:, k, :].ravel())
    return Wk, Dk


def dense_kgrad_factored(X, grid, factors, outputscale):
    """Dense B K_UU B^T without forming K_UU (grids too large for
    kuu_dense).  Every row of B is a tensor product of per-dimension
    stencils and K_UU = s_f^2 K_1 (x) ... (x) K_d, so each entry factors over
    dimensions:
      (B K_UU B^T)[(i,c), (j,c')] = s_f^2 prod_k (a_k K_k b_k^T)[i, j],
    with a_k = dW_k if c = k + 1 else W_k (rows; c = 0 value, c = p + 1 the
    derivative in dimension p) and b_k likewise for c'.  `factors` are the
    K_k (any symmetric m_k x m_k matrices, e.g. dK_k / dlog l_k in one
    dimension).  Block order [values; d/dx_1; ...]."""
    X = np.asarray(X, np.float64)
    n, d = X.shape
    blocks = []
    for k in range(d):
        Wk, Dk = interp_matrix_1d(X, grid, k)
        Kk = factors[k]
        WK, DK = Wk @ Kk, Dk @ Kk
        blocks.append({(0, 0): WK @ Wk.T, (1, 0): DK @ Wk.T, (0, 1): WK @ Dk.T,
                       (1, 1): DK @ Dk.T})
    out = np.empty((n * (d + 1), n * (d + 1)))
    for c in range(d + 1):
        for c2 in range(d + 1):
            T = np.full((n, n), float(outputscale) ** 2)
            for k in range(d):
                T *= blocks[k][(int(c == k + 1), int(c2 == k + 1))]
            out[c * n:(c + 1) * n, c2 * n:(c2 + 1) * n] = T
    return out


def noise_diag(n, d, noise_value, noise_grad):
    """Diagonal of the noise term: sigma_v^2 on value rows, sigma_g^2 on gradient rows."""
    return np.concatenate([np.full(n, float(noise_value)), np.full(n * d, float(noise_grad))])


class DSKI:
    """The D-SKI operator K~ = B K_UU B^T + diag(noise) for fixed data X."""

    def __init__(self, X, grid, lengthscale, outputscale, noise_value, noise_grad):
        self.X = np.asarray(X, np.float64)
        self.n, self.d = self.X.shape
        self.N = self.n * (self.d + 1)
        self.grid = grid
        self.ell = np.asarray(lengthscale, np.float64)
        self.sf = float(outputscale)
        self.B = interp_matrix(self.X, grid)
        self.noise = noise_diag(self.n, self.d, noise_value, noise_grad)

    def kgrad_mvm(self, V):
        """K^grad_SKI V = B K_UU B^T V (no noise)."""
        V = np.asarray(V, np.float64)
        vec = V.ndim == 1
        V2 = V.reshape(self.N, -1)
        G = self.B.T @ V2
        H = kuu_apply(self.grid, self.ell, self.sf, G)
        out = self.B @ H
        return out.ravel() if vec else out

    def mvm(self, V):
        """K~ V = B K_UU B^T V + noise * V (the D-SKI MVM of Sec. 3.1)."""
        V = np.asarray(V, np.float64)
        nz = self.noise if V.ndim == 1 else self.noise[:, None]
        return self.kgrad_mvm(V) + nz * V

    def abs_mvm(self, V):
        """|B| K_UU |B|^T |V| + noise * |V|: the same product with every term
        replaced by its absolute value (K_UU >= 0 elementwise for the SE
        kernel).  The standard rounding-error bound of a product evaluated
        term by term in precision u is |fl(K~ v) - K~ v| <= gamma |B| K_UU
        |B|^T |v| (Higham, Accuracy and Stability of Numerical Algorithms,
        2nd ed., Sec. 3.5); this supplies the right-hand side."""
        V = np.abs(np.asarray(V, np.float64))
        vec = V.ndim == 1
        V2 = V.reshape(self.N, -1)
        Ba = abs(self.B)
        out = Ba @ kuu_apply(self.grid, self.ell, self.sf, Ba.T @ V2)
        out = out + self.noise[:, None] * V2
        return out.ravel() if vec else out

    def dense_kgrad(self):
        """Dense B K_UU B^T (small grids)."""
        Bd = self.B.toarray()
        return Bd @ kuu_dense(self.grid, self.ell, self.sf) @ Bd.T

    def dense(self):
        return self.dense_kgrad() + np.diag(self.noise)

    def kgrad_diag(self):
        """diag(B K_UU B^T): each row's stencil block of K_UU (Sec. 3.3)."""
        B = self.B.tocsr()
        out = np.empty(self.N)
        facs = [kfactor(self.grid, k, self.ell[k]) for k in range(self.d)]
        for i in range(self.N):
            cols = B.indices[B.indptr[i]:B.indptr[i + 1]]
            vals = B.data[B.indptr[i]:B.indptr[i + 1]]
            idx = np.array(np.unravel_index(cols, self.grid.m))      # d x nnz
            blk = np.ones((len(cols), len(cols)))
            for k in range(self.d):
                blk = blk * facs[k][np.ix_(idx[k], idx[k])]
            out[i] = self.sf**2 * vals @ blk @ vals
        return out

    def kgrad_row(self, j):
        """Row j of B K_UU B^T: B (K_UU B[j]^T) (Sec. 3.3)."""
        bj = self.B.getrow(j).toarray().ravel()
        h = kuu_apply(self.grid, self.ell, self.sf, bj[:, None])[:, 0]
        return self.B @ h
