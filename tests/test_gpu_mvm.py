"""GPU parity of the D-SKI MVM (Sec. 3.1) against the FP64 oracle.

FP64 and FP64_TC modes must match to 1e-10 relative (2-norm per column); the
mixed modes to u * cond, with u the unit roundoff of the mode (2^-24 for
FP32 / 3xTF32, 2^-11 for plain TF32) and cond = || |B| K_UU |B|^T |v| || /
||K~ v|| the condition number of evaluating the product (see mvm_tolerance).
Every column is also checked element by element: |got_i - ref_i| <=
gamma_K (|B| K_UU |B|^T |v| + noise |v|)_i, the componentwise bound with K
the longest rounding chain of the product (see elem_tolerance), so a wrong
row block cannot hide under a column norm.  Cases span several tiles and
ragged tails: d = 1, 2, 3, odd grid sizes, n = 1, s not a multiple of the
column block, points on grid lines, and out-of-grid rejection.
"""
import numpy as np
import pytest

from synth import workloads as W
from tests._gpu_helpers import (gpu_op, oracle_op, need_gpu, rel, problem_1d, torch,
                                mvm_tolerance, check_mvm, elem_err, elem_tolerance)

pytestmark = pytest.mark.gpu

CASES = [
    ("1d", lambda: problem_1d(300, m=37)),
    ("2d", lambda: W.small2d(500, m=21, seed=3)),
    ("3d", lambda: W.small3d(300, m=11, seed=4)),
    ("sine2d", lambda: W.sine2d()),
]


@pytest.mark.parametrize("prec", ["fp64", "mixed_3xtf32", "mixed_tf32"])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("s", [1, 3, 9])
def test_mvm_parity(name, make, prec, s):
    need_gpu()
    p = make()
    op = gpu_op(p, prec)
    orc = oracle_op(p)
    rng = np.random.default_rng(11)
    V = rng.normal(size=(s, orc.N))
    got = op.mvm(torch.tensor(V, device="cuda")).double().cpu().numpy()
    ref = orc.mvm(V.T).T
    for q in range(s):
        check_mvm(orc, V[q], got[q], prec, ref=ref[q])
    op.close()


# FP64_TC takes the tensor cores for modes of at least 64 nodes (the FP64
# units below); these grids mix both, with two 128-row tiles and ragged
# tails in j and r, contraction splits of 2..5, and an operand of one row
TC_CASES = [
    ("1d-m64", lambda: problem_1d(300, m=64)),
    ("2d-136x72", lambda: dict(W.small2d(700, m=24, seed=5), m=(136, 72))),
    ("3d-64x16x24", lambda: dict(W.small3d(400, m=16, seed=6), m=(64, 16, 24))),
    ("2d-24x32-fp64-units", lambda: dict(W.small2d(700, m=24, seed=5), m=(24, 32))),
    ("sine2d-64", lambda: dict(W.sine2d(), m=(64, 64))),
]


@pytest.mark.parametrize("name,make", TC_CASES, ids=[c[0] for c in TC_CASES])
@pytest.mark.parametrize("s", [1, 5])
def test_mvm_fp64_tc_parity(name, make, s):
    """FP64_TC: FP64 scatter/gather with digit-split BF16 tensor-core mode
    products; grids with every m_k a multiple of 8 (several 128-row tiles
    and ragged tails in j and r)."""
    need_gpu()
    p = make()
    op = gpu_op(p, "fp64_tc")
    orc = oracle_op(p)
    V = np.random.default_rng(12).normal(size=(s, orc.N))
    got = op.mvm(torch.tensor(V, device="cuda")).cpu().numpy()
    ref = orc.mvm(V.T).T
    for q in range(s):
        check_mvm(orc, V[q], got[q], "fp64_tc", ref=ref[q])
    op.close()


def test_mvm_single_point_and_grid_line():
    need_gpu()
    # one point exactly on a grid line in x (fraction 0) and one interior
    p = W.small2d(2, m=12, seed=1)
    lo, hi, m = p["lo"][0], p["hi"][0], p["m"][0]
    h = (hi - lo) / (m - 1)
    X = p["X"].copy()
    X[0, 0] = lo + 5 * h
    p["X"] = X
    for n in (1, 2):
        q = dict(p)
        q["X"] = X[:n].copy()
        op = gpu_op(q, "fp64")
        orc = oracle_op(q)
        V = np.random.default_rng(0).normal(size=orc.N)
        got = op.mvm(torch.tensor(V, device="cuda")).cpu().numpy()
        assert rel(got, orc.mvm(V)) <= 1e-12
        check_mvm(orc, V, got, "fp64")
        op.close()


def test_mvm_deterministic():
    need_gpu()
    p = W.small3d(400, m=10, seed=9)
    for prec in ("fp64", "mixed_3xtf32"):
        op = gpu_op(p, prec)
        V = torch.randn(4, op.N, device="cuda", dtype=op.dtype)
        a = op.mvm(V)
        b = op.mvm(V)
        assert torch.equal(a, b)
        op.close()


def test_mvm_out_of_grid_rejected():
    need_gpu()
    from paper_1810_12283_gb300 import DskiError
    p = W.small2d(50, m=12, seed=2)
    p["X"] = p["X"].copy()
    p["X"][7, 1] = p["hi"][1] - 0.5 * (p["hi"][1] - p["lo"][1]) / (p["m"][1] - 1)
    with pytest.raises(DskiError) as e:
        gpu_op(p, "fp64")
    assert e.value.status == "OUT_OF_GRID"


def test_mvm_terrain_sampled_rows():
    """Full-size terrain operator (n = 100,000, 256^2 grid): compare sampled
    output rows with the oracle's sparse rows B[i] K_UU B^T v."""
    need_gpu()
    p = W.terrain2d()
    orc = oracle_op(p)
    v = np.random.default_rng(5).normal(size=orc.N)
    from oracle.dski import kuu_apply
    h = kuu_apply(orc.grid, orc.ell, orc.sf, (orc.B.T @ v)[:, None])[:, 0]
    rows = np.random.default_rng(6).choice(orc.N, 2000, replace=False)
    ref = orc.B[rows] @ h + orc.noise[rows] * v[rows]
    habs = kuu_apply(orc.grid, orc.ell, orc.sf, (abs(orc.B).T @ np.abs(v))[:, None])[:, 0]
    absr = abs(orc.B[rows]) @ habs + orc.noise[rows] * np.abs(v[rows])
    for prec in ("fp64", "mixed_3xtf32", "fp64_tc"):
        if prec == "mixed_3xtf32":
            tol = max(1e-6, 2.0**-24 * np.linalg.norm(absr) / np.linalg.norm(ref))
        else:
            tol = 1e-10
        etol = elem_tolerance(orc, prec)
        op = gpu_op(p, prec)
        got = op.mvm(torch.tensor(v, device="cuda")).double().cpu().numpy()[rows]
        assert rel(got, ref) <= tol, (prec, rel(got, ref), tol)
        assert elem_err(got, ref, absr) <= etol, (prec, elem_err(got, ref, absr), etol)
        op.close()
