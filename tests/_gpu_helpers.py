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


# unit roundoff of the arithmetic each mode evaluates the product in
UNIT_ROUNDOFF = {"fp64": 2.0**-53, "mixed_3xtf32": 2.0**-24, "mixed_tf32": 2.0**-11,
                 "fp64_tc": 2.0**-40}


def mvm_tolerance(orc, v, prec):
    """Normwise tolerance for one MVM column, derived from the arithmetic.

    FP64 mode: 1e-10 relative.  Other modes: u * ||abs|| / ||K~ v|| (the
    condition number of evaluating the product term by term times the unit
    roundoff of the mode), never below 1e-6 (FP32 modes) or 1e-10 (FP64_TC,
    whose digit-split mode products carry ~2^-61 error relative to the
    operands' row maxima; u = 2^-40 leaves a wide margin).  D-SKI gradient rows cancel
    terms of size ~1/h against results of size ~1/l, so this condition
    number reaches ~1e5 on fine grids; the bound is the textbook
    normwise one (Higham, Sec. 3.5) with gamma_k replaced by u."""
    if prec == "fp64":
        return 1e-10
    a = orc.abs_mvm(v)
    r = orc.mvm(v)
    floor = 1e-10 if prec == "fp64_tc" else 1e-6
    return max(floor, UNIT_ROUNDOFF[prec] * np.linalg.norm(a) / np.linalg.norm(r))
