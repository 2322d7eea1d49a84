"""GB300 D-SKI: the derivative structured-kernel-interpolation MVM of
Eriksson et al., "Scaling Gaussian Process Regression with Derivatives"
(NeurIPS 2018, Sec. 3.1), with the pivoted-Cholesky-preconditioned CG,
stochastic-Lanczos log determinant and marginal-likelihood gradient it drives
(Sec. 2, Sec. 3.3, Eq. 1).

This module is the thin Python binding of the C ABI declared in
``include/dski.h``: it marshals torch CUDA tensors (device memory, streams)
into the library's calls and nothing else.  Every step of the computation
runs in the CUDA library ``libdski.so``; importing fails loudly when the
library has not been built.
"""
import ctypes as C

import torch

from . import _lib
from ._lib import DskiError, PREC, INTERP, KUU

__all__ = ["DSKI", "Preconditioner", "DskiError", "PREC", "INTERP", "KUU", "mll_function", "launch_count"]


def _stream_ptr(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _dptr(t):
    return C.c_void_p(t.data_ptr())


class Preconditioner:
    """Truncated pivoted Cholesky preconditioner M = D + L L^T (Sec. 3.3)."""

    def __init__(self, handle, ptr, rank):
        self._owner = handle
        self.ptr = ptr
        self.rank = rank

    def logdet(self):
        """log|M| (Sylvester's identity through the CholeskyQR factor)."""
        return float(_lib.load().pivchol_logdet(self.ptr))

    def export(self):
        """(L, pivots): L as an (rank, N) float64 CUDA tensor (row k = column k
        of the factor, caller block order) and the pivot rows chosen."""
        op = self._owner
        L = torch.empty(max(self.rank, 1), op.N, dtype=torch.float64, device=op.device)
        piv = (C.c_int * max(self.rank, 1))()
        _lib.check(_lib.load().pivchol_export(self.ptr, _dptr(L), piv))
        return L[:self.rank], list(piv)[:self.rank]

    def close(self):
        if self.ptr:
            _lib.load().pivchol_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DSKI:
    """D-SKI operator K~ = [W; dW] K_UU [W; dW]^T + diag(noise) on a regular grid.

    X: (n, d) float64 CUDA tensor of points.  ``interp`` picks the stencil of
    W and dW: "cubic" (Keys, 4^d nodes per row) or "quintic" (the paper's
    six-point kernel, 6^d nodes per row).  ``kuu`` picks how the Kronecker
    factors of K_UU are applied: "dense" or "fft" (Toeplitz factors through
    circulant embedding and FP64 FFTs; FP64 and FP64_TC modes).  Vectors are
    length N = n(d+1)
    in block order [values; d/dx_1; ...; d/dx_d] (columns of an (N, s)
    tensor stored column-major, i.e. pass ``V.T.contiguous().T`` or an
    (s, N) tensor's transpose -- the helpers below take (N,) or (s, N)).
    """

    def __init__(self, X, grid_m, grid_lo, grid_hi, lengthscale, outputscale=1.0,
                 noise_value=1e-4, noise_grad=None, prec="fp64", stream=None,
                 interp="cubic", kuu="dense"):
        lib = _lib.load()
        if not (isinstance(X, torch.Tensor) and X.is_cuda):
            raise TypeError("X must be a CUDA tensor")
        X = X.to(torch.float64).contiguous()
        n, d = X.shape
        self.n, self.d, self.N = n, d, n * (d + 1)
        self.prec = prec
        self.interp = interp
        self.kuu = kuu
        self.dtype = torch.float64 if prec in ("fp64", "fp64_tc") else torch.float32
        self.device = X.device
        self.stream = stream
        ng = noise_value if noise_grad is None else noise_grad
        self.noise_ratio = float(ng) / float(noise_value)
        self._m = (C.c_int * d)(*[int(v) for v in grid_m])
        self._lo = (C.c_double * d)(*[float(v) for v in grid_lo])
        self._hi = (C.c_double * d)(*[float(v) for v in grid_hi])
        ell = list(lengthscale) if hasattr(lengthscale, "__len__") else [lengthscale] * d
        self._ell = (C.c_double * d)(*[float(v) for v in ell])
        p = _lib.DskiParams(n, d, self._m, self._lo, self._hi, self._ell, float(outputscale),
                            float(noise_value), float(ng), PREC[prec], INTERP[interp], KUU[kuu])
        h = C.c_void_p()
        _lib.check(lib.dski_create(C.byref(h), C.byref(p), _dptr(X), _stream_ptr(stream)))
        self.h = h

    # -- helpers -------------------------------------------------------------
    def _cols(self, v, dtype):
        """(N,) or (s, N) -> contiguous (s, N) tensor of dtype on our device."""
        if v.dim() == 1:
            v = v[None, :]
        if v.shape[-1] != self.N:
            raise ValueError(f"expected trailing size N={self.N}, got {tuple(v.shape)}")
        return v.to(device=self.device, dtype=dtype).contiguous()

    def close(self):
        if getattr(self, "h", None):
            _lib.load().dski_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls -----------------------------------------------------------------
    def set_hypers(self, lengthscale, outputscale, noise_value, noise_grad=None):
        ng = noise_value if noise_grad is None else noise_grad
        ell = list(lengthscale) if hasattr(lengthscale, "__len__") else [lengthscale] * self.d
        arr = (C.c_double * self.d)(*[float(v) for v in ell])
        _lib.check(_lib.load().dski_set_hypers(self.h, arr, float(outputscale),
                                               float(noise_value), float(ng)))

    def mvm(self, v, out=None):
        """K~ v for v of shape (N,) or (s, N) (each row one column of the C-ABI's N x s)."""
        squeeze = v.dim() == 1
        V = self._cols(v, self.dtype)
        s = V.shape[0]
        if out is None:
            res = torch.empty_like(V)
            _lib.check(_lib.load().dski_mvm(self.h, _dptr(V), _dptr(res), s))
            return res[0] if squeeze else res
        if (out.dtype != self.dtype or not out.is_contiguous() or out.numel() != V.numel()
                or out.device != V.device):
            raise ValueError("out must be a contiguous tensor of the operator's dtype and size")
        _lib.check(_lib.load().dski_mvm(self.h, _dptr(V), _dptr(out), s))
        return out

    def pivchol(self, rank):
        pc = C.c_void_p()
        got = C.c_int()
        _lib.check(_lib.load().pivchol_build(self.h, int(rank), C.byref(pc), C.byref(got)))
        return Preconditioner(self, pc, got.value)

    def solve(self, b, pc=None, rtol=1e-8, maxit=10000, x0=None, allow_not_converged=False):
        """Solve K~ x = b.  Returns (x, iters list, relres list)."""
        squeeze = b.dim() == 1
        B = self._cols(b, torch.float64)
        s = B.shape[0]
        X = torch.zeros_like(B) if x0 is None else self._cols(x0, torch.float64).clone()
        it = (C.c_int * s)()
        rr = (C.c_double * s)()
        allow = (-4,) if allow_not_converged else ()
        _lib.check(_lib.load().dski_pcg_solve(self.h, pc.ptr if pc is not None else None,
                                              _dptr(B), _dptr(X), s, float(rtol), int(maxit),
                                              it, rr), allow)
        return (X[0] if squeeze else X), list(it), list(rr)

    def profile_start(self):
        """Start the per-stage device timers (dski_profile mode 1)."""
        _lib.check(_lib.load().dski_profile(self.h, 1, None, None, None, None))

    def profile_stop(self):
        """Stop the timers; returns {stage: (ms, launches, timed launches)}
        and a truncated flag (ms covers the timed launches only)."""
        ms = (C.c_double * _lib.NSTAGES)()
        la = (C.c_longlong * _lib.NSTAGES)()
        tl = (C.c_longlong * _lib.NSTAGES)()
        tr = C.c_int()
        _lib.check(_lib.load().dski_profile(self.h, 0, ms, la, tl, C.byref(tr)))
        return ({name: (ms[k], la[k], tl[k]) for k, name in enumerate(_lib.STAGES)},
                bool(tr.value))

    def logdet(self, pc, probes=16, depth=30, seed=777):
        ld = C.c_double()
        se = C.c_double()
        _lib.check(_lib.load().dski_logdet_slq(self.h, pc.ptr, int(probes), int(depth),
                                               C.c_uint64(seed), C.byref(ld), C.byref(se)))
        return ld.value, se.value

    def mll_grad(self, y, pc, probes=16, seed=777, rtol=None, maxit=100000):
        """Log marginal likelihood of Eq. 1 and its gradient (log l_1..d,
        log s_f, log s_n).  rtol, maxit: the batched PCG's stopping rule
        (defaults 1e-8 and 100,000: dski_mll_grad; otherwise
        dski_mll_grad_tol)."""
        Y = self._cols(y, torch.float64)
        mll = C.c_double()
        g = (C.c_double * (self.d + 2))()
        if rtol is None and maxit == 100000:
            _lib.check(_lib.load().dski_mll_grad(self.h, pc.ptr, _dptr(Y), int(probes),
                                                 C.c_uint64(seed), C.byref(mll), g))
        else:
            _lib.check(_lib.load().dski_mll_grad_tol(self.h, pc.ptr, _dptr(Y), int(probes),
                                                     C.c_uint64(seed),
                                                     float(1e-8 if rtol is None else rtol),
                                                     int(maxit), C.byref(mll), g))
        return mll.value, list(g)

    def set_wait_budget(self, polls):
        """Test aid: cap the first mbarrier wait of the tensor-core mode
        products at `polls` polls (0: gives up at once; < 0: default)."""
        _lib.check(_lib.load().dski_set_wait_budget(self.h, int(polls)))

    def predict(self, alpha, Xs, pc=None, with_grad=True, variance=True):
        """Mean (and gradient, block order) at the test points Xs (n* x d
        CUDA float64) from alpha = K~^-1 y; with pc, the preconditioner
        variance estimate as well.  Returns (mean, var or None)."""
        Xs = Xs.to(device=self.device, dtype=torch.float64).contiguous()
        if Xs.dim() != 2 or Xs.shape[1] != self.d:
            raise ValueError(f"Xs must be n* x {self.d}")
        ns = Xs.shape[0]
        A = None if alpha is None else self._cols(alpha, torch.float64)
        mean = None
        if A is not None:
            mean = torch.empty(ns * (self.d + 1) if with_grad else ns, device=self.device,
                               dtype=torch.float64)
        var = torch.empty(ns, device=self.device, dtype=torch.float64) if (pc is not None and variance) else None
        _lib.check(_lib.load().dski_predict(self.h, pc.ptr if pc is not None else None,
                                            _dptr(A) if A is not None else None, _dptr(Xs), ns,
                                            1 if with_grad else 0,
                                            _dptr(mean) if mean is not None else None,
                                            _dptr(var) if var is not None else None))
        return mean, var

    def predict_variance_cv(self, Xs, pc, probes=64, seed=777, rtol=1e-8, maxit=20000):
        """Unbiased predictive variance (randomized estimator with the
        preconditioner estimate as control variate) at Xs (n* x d)."""
        Xs = Xs.to(device=self.device, dtype=torch.float64).contiguous()
        var = torch.empty(Xs.shape[0], device=self.device, dtype=torch.float64)
        _lib.check(_lib.load().dski_predict_var_cv(self.h, pc.ptr, _dptr(Xs), Xs.shape[0],
                                                   int(probes), C.c_uint64(seed), float(rtol),
                                                   int(maxit), _dptr(var)))
        return var


def launch_count():
    """Kernels the CUDA library has launched in this process."""
    return int(_lib.load().dski_launch_count())


def mll_function(*args, **kwargs):
    from .autograd import mll_function as f
    return f(*args, **kwargs)


def solve_batch(ops, pcs, bs, rtol=1e-8, maxit=10000, x0s=None, allow_failed=False, cluster=0):
    """Solve K~_i x_i = b_i for many independent systems in one persistent
    launch (dski_pcg_solve_batch): ops[i] a DSKI (FP64 or FP64_TC), pcs[i]
    its Preconditioner or None, bs[i] its N_i right-hand side (cuda FP64).
    Returns (xs, iters, relres, status, seconds) with per-system lists;
    status is "OK" or the failure's name.  allow_failed: return the
    outputs of systems that did not converge or broke down instead of
    raising.  cluster: CTAs per system (1, 2, 4 or 8; 0: the default)."""
    k = len(ops)
    if not (len(pcs) == len(bs) == k) or k == 0:
        raise ValueError("solve_batch: ops, pcs and bs must be non-empty and of equal length")
    Bs = [torch.as_tensor(b, dtype=torch.float64, device="cuda").contiguous() for b in bs]
    if x0s is None:
        Xs = [torch.zeros_like(b) for b in Bs]
    else:
        Xs = [torch.as_tensor(x, dtype=torch.float64, device="cuda").clone().contiguous()
              for x in x0s]
    vp = C.c_void_p
    H = (vp * k)(*[op.h for op in ops])
    P = (vp * k)(*[(pc.ptr if pc is not None else None) for pc in pcs])
    Bp = (vp * k)(*[b.data_ptr() for b in Bs])
    Xp = (vp * k)(*[x.data_ptr() for x in Xs])
    it = (C.c_int * k)()
    rr = (C.c_double * k)()
    stt = (C.c_int * k)()
    sec = (C.c_double * k)()
    torch.cuda.synchronize()
    rc = _lib.load().dski_pcg_solve_batch(k, H, P, Bp, Xp, float(rtol), int(maxit), int(cluster),
                                          it, rr, stt, sec)
    _lib.check(rc, (-4, -5) if allow_failed else ())
    status = [_lib.STATUS.get(v, str(v)) for v in stt]
    return Xs, list(it), list(rr), status, list(sec)

