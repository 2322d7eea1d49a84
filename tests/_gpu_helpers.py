"""Shared helpers for the GPU parity tests: build the CUDA operator and the
oracle operator from the same seeded synthetic problem."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def gpu_op(p, prec="fp64"):
    from paper_1810_12283_gb300 import DSKI
    X = torch.tensor(p["X"], dtype=torch.float64, device="cuda")
    return DSKI(X, p["m"], p["lo"], p["hi"], p["ell"], p["sf"], p["noise_value"],
                p["noise_grad"], prec=prec, interp=p.get("interp", "cubic"),
                kuu=p.get("kuu", "dense"))


def oracle_op(p):
    from oracle.dski import DSKI as ODSKI, Grid
    return ODSKI(p["X"], Grid(p["m"], p["lo"], p["hi"], p.get("interp", "cubic")), p["ell"],
                 p["sf"], p["noise_value"], p["noise_grad"])


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def problem_1d(n, m=20, seed=0, ell=0.15):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, (n, 1))
    return dict(X=X, y=rng.normal(size=2 * n), m=(m,), lo=(-0.25,), hi=(1.25,), ell=(ell,),
                sf=1.3, noise_value=1e-3, noise_grad=2e-3, name=f"line1d-n{n}")


# unit roundoff of the arithmetic each mode evaluates the product in.  FP64_TC
# forms its mode products from 62-bit integer digits with exact accumulation
# (error <= m 2^-60 max|K_j| max|X_r| per output, below FP64's
# gamma_m sum |K_ji||X_ri| bound up to the row-max ratio) and rounds each
# output once to double, so it is held to FP64's bar.
UNIT_ROUNDOFF = {"fp64": 2.0**-53, "fp64_tc": 2.0**-53, "mixed_3xtf32": 2.0**-24,
                 "mixed_tf32": 2.0**-11}
# per-term representation error for the componentwise bound: the 3xTF32
# split represents an FP32 operand as hi + lo to 2^-22, plain TF32 to 2^-11.
# FP64_TC's d = 2 cubic scatter forms its stencil products in double-float
# arithmetic (FP32 hi + lo pairs; FMA exact products and TwoSum sums): each
# step is exact up to the dropped lo x lo term and the FP32 rounding of the
# lo accumulator, each <= 2^-48 of the magnitudes combined, so its chain
# bound takes u = 2^-47 (the FP64 parts are covered a fortiori).
UNIT_ELEM = {"fp64": 2.0**-53, "fp64_tc": 2.0**-47, "mixed_3xtf32": 2.0**-22,
             "mixed_tf32": 2.0**-11}


def mvm_tolerance(orc, v, prec):
    """Normwise tolerance for one MVM column, derived from the arithmetic.

    FP64 and FP64_TC: 1e-10 relative.  Mixed modes: u * ||abs|| / ||K~ v||
    (the condition number of evaluating the product term by term times the
    unit roundoff of the mode), never below 1e-6.  D-SKI gradient rows cancel
    terms of size ~1/h against results of size ~1/l, so this condition number
    reaches ~1e5 on fine grids; the bound is the textbook normwise one
    (Higham, Sec. 3.5) with gamma_k replaced by u."""
    if prec in ("fp64", "fp64_tc"):
        return 1e-10
    a = orc.abs_mvm(v)
    r = orc.mvm(v)
    return max(1e-6, UNIT_ROUNDOFF[prec] * np.linalg.norm(a) / np.linalg.norm(r))


def chain_length(orc):
    """Longest chain of roundings one output element of the D-SKI MVM goes
    through: the scatter sum at a grid node ((d+1) S^d terms per point in
    the cells around it), the d mode products (m_k terms each), the gather
    (S^d terms), the weights (2d roundings) and the noise term."""
    g = orc.grid
    S, lead = g.stencil
    d = g.d
    X = orc.X
    cells = np.zeros(tuple(g.m), np.int64)
    idx = tuple(np.floor((X[:, k] - g.lo[k]) / g.h[k]).astype(np.int64) for k in range(d))
    np.add.at(cells, idx, 1)
    per_node = cells.max() * S**d
    return (d + 1) * per_node + sum(g.m) + S**d + 2 * d + 2


def elem_tolerance(orc, prec):
    """Componentwise bound |fl(K~ v)_i - (K~ v)_i| <= gamma_K abs_i with
    abs = |B| K_UU |B|^T |v| + noise |v| and K the chain length
    (Higham, Sec. 3.5), doubled because both the GPU and the oracle round.
    gamma_K = K u / (1 - K u) holds for K u < 1; for plain TF32 (u = 2^-11)
    on long chains K u exceeds that, and the first-order bound 2 K u (no
    better than the trivial one) is used."""
    K = chain_length(orc)
    u = UNIT_ELEM[prec]
    if K * u < 0.5:
        return 2.0 * K * u / (1.0 - K * u)
    return 2.0 * K * u


def elem_err(got, ref, absr):
    """max_i |got_i - ref_i| / abs_i (rows with abs_i = 0 must match exactly)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    absr = np.asarray(absr, np.float64)
    diff = np.abs(got - ref)
    zero = absr == 0
    if np.any(diff[zero] != 0):
        return np.inf
    return float(np.max(diff[~zero] / absr[~zero])) if np.any(~zero) else 0.0


def check_mvm(orc, v, got, prec, ref=None):
    """Normwise and componentwise check of one MVM column against the oracle;
    returns (normwise error, its tolerance, componentwise error, its bound)."""
    ref = orc.mvm(v) if ref is None else ref
    tol = mvm_tolerance(orc, v, prec)
    e = rel(got, ref)
    absr = orc.abs_mvm(v)
    ee = elem_err(got, ref, absr)
    etol = elem_tolerance(orc, prec)
    assert e <= tol, ("normwise", prec, e, tol)
    assert ee <= etol, ("componentwise", prec, ee, etol)
    return e, tol, ee, etol
