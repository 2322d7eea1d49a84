"""GPU parity of the quintic D-SKI operator (the paper's six-point kernel,
6^d weights per row of W and dW, Sec. 3.1) against the FP64 oracle.

The same bars as the cubic path: the MVM in every precision mode (FP64 and
FP64_TC 1e-10; the others u * cond, see mvm_tolerance; and element by
element within the componentwise bound, see elem_tolerance) for d = 1, 2, 3
and s = 1, 3, 9; pivoted Cholesky pivots and factor (1e-10); the PCG solve through the
fused CG path and the grid-form preconditioner against the dense direct
solve; the predictive mean; and the quintic stencil's grid bounds
(2 <= floor(t) <= m - 4, m >= 6)."""
import numpy as np
import pytest

from synth import workloads as W
from tests._gpu_helpers import (gpu_op, oracle_op, need_gpu, rel, problem_1d, torch,
                                check_mvm)

pytestmark = pytest.mark.gpu


def Q(p):
    q = dict(p)
    q["interp"] = "quintic"
    return q


CASES = [
    ("1d", lambda: Q(problem_1d(300, m=37))),
    ("2d", lambda: Q(W.small2d(500, m=21, seed=3))),
    ("3d", lambda: Q(W.small3d(300, m=14, seed=4))),
    ("sine2d", lambda: Q(W.sine2d())),
]


@pytest.mark.parametrize("prec", ["fp64", "mixed_3xtf32", "mixed_tf32"])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("s", [1, 3, 9])
def test_quintic_mvm_parity(name, make, prec, s):
    need_gpu()
    p = make()
    op = gpu_op(p, prec)
    orc = oracle_op(p)
    assert orc.B[:orc.n].getnnz(axis=1).max() > 4 ** orc.d   # the wider stencil is in use
    V = np.random.default_rng(21).normal(size=(s, orc.N))
    got = op.mvm(torch.tensor(V, device="cuda")).double().cpu().numpy()
    ref = orc.mvm(V.T).T
    for q in range(s):
        check_mvm(orc, V[q], got[q], prec, ref=ref[q])
    op.close()


TC_CASES = [
    ("2d-136x72", lambda: Q(dict(W.small2d(700, m=24, seed=5), m=(136, 72)))),
    ("3d-64x16x24", lambda: Q(dict(W.small3d(400, m=16, seed=6), m=(64, 16, 24)))),
]


@pytest.mark.parametrize("name,make", TC_CASES, ids=[c[0] for c in TC_CASES])
@pytest.mark.parametrize("s", [1, 5])
def test_quintic_mvm_fp64_tc_parity(name, make, s):
    need_gpu()
    p = make()
    op = gpu_op(p, "fp64_tc")
    orc = oracle_op(p)
    V = np.random.default_rng(22).normal(size=(s, orc.N))
    got = op.mvm(torch.tensor(V, device="cuda")).cpu().numpy()
    ref = orc.mvm(V.T).T
    for q in range(s):
        check_mvm(orc, V[q], got[q], "fp64_tc", ref=ref[q])
    op.close()


@pytest.mark.parametrize("make,rank", [(lambda: Q(W.small2d(60, m=16, seed=2)), 20),
                                        (lambda: Q(W.small3d(40, m=12, seed=3)), 25)],
                         ids=["2d", "3d"])
def test_quintic_pivoted_cholesky_parity(make, rank):
    need_gpu()
    from oracle.solve import QRPreconditioner, pivoted_cholesky
    p = make()
    op = gpu_op(p, "fp64")
    orc = oracle_op(p)
    pc = op.pivchol(rank)
    Lg, piv = pc.export()
    Lo, piv_o, _ = pivoted_cholesky(orc.kgrad_diag(), orc.kgrad_row, rank)
    assert piv == piv_o
    assert rel(Lg.cpu().numpy().T, Lo) <= 1e-10
    ld = QRPreconditioner(Lo, orc.noise).logdet()
    assert abs(pc.logdet() - ld) <= 1e-10 * abs(ld)
    pc.close()
    op.close()


@pytest.mark.parametrize("prec", ["fp64", "fp64_tc"])
def test_quintic_pcg_matches_direct_solve(prec):
    """Fused FP64 CG path (d = 2, s <= 4) with the grid-form preconditioner
    (M < N); FP64_TC with a 64-node mode on the tensor cores."""
    need_gpu()
    p = Q(dict(W.small2d(2000, m=24, seed=7, nv=1e-2, ng=1e-2), m=(56, 64)))
    op = gpu_op(p, prec)
    orc = oracle_op(p)
    A = orc.dense()
    pc = op.pivchol(20)
    rng = np.random.default_rng(4)
    B = np.stack([p["y"], rng.normal(size=orc.N)])
    # rtol 1e-7: this system's attainable FP64 residual is near 1e-8
    x, it, rr = op.solve(torch.tensor(B, device="cuda"), pc, rtol=1e-7, maxit=20000)
    x = x.cpu().numpy()
    for q in range(2):
        assert rr[q] <= 1e-7
        assert np.linalg.norm(B[q] - A @ x[q]) / np.linalg.norm(B[q]) <= 1.5e-7
        xd = np.linalg.solve(A, B[q])
        assert np.linalg.norm(A @ (x[q] - xd)) / np.linalg.norm(B[q]) <= 2e-7
    pc.close()
    op.close()


def test_quintic_predictive_mean():
    need_gpu()
    from oracle.predict import dski_mean
    p = Q(W.sine2d())
    orc = oracle_op(p)
    alpha = np.random.default_rng(5).normal(size=orc.N)
    rng = np.random.default_rng(6)
    Xs = rng.uniform(0.02, 0.98, (41, 2))
    want = dski_mean(orc, alpha, Xs)
    op = gpu_op(p, "fp64")
    mean, _ = op.predict(torch.tensor(alpha, device="cuda"), torch.tensor(Xs, device="cuda"))
    assert rel(mean.cpu().numpy(), want) <= 1e-12
    op.close()


def test_quintic_grid_bounds():
    need_gpu()
    from paper_1810_12283_gb300 import DskiError
    p = W.small2d(40, m=16, seed=2)
    h0 = (p["hi"][0] - p["lo"][0]) / (p["m"][0] - 1)
    X = p["X"].copy()
    X[3, 0] = p["lo"][0] + 1.5 * h0          # floor(t) = 1: cubic yes, quintic no
    p["X"] = X
    gpu_op(p, "fp64").close()
    with pytest.raises(DskiError) as e:
        gpu_op(Q(p), "fp64")
    assert e.value.status == "OUT_OF_GRID"
    X[3, 0] = p["lo"][0] + 2.25 * h0         # floor(t) = 2: the first quintic cell
    op = gpu_op(Q(p), "fp64")
    orc = oracle_op(Q(p))
    v = np.random.default_rng(0).normal(size=orc.N)
    assert rel(op.mvm(torch.tensor(v, device="cuda")).cpu().numpy(), orc.mvm(v)) <= 1e-10
    op.close()
    q = Q(W.small2d(10, m=5, seed=1))
    q["m"] = (5, 8)
    with pytest.raises(DskiError) as e:
        gpu_op(q, "fp64")
    assert e.value.status == "ARG"


def test_quintic_slq_and_mll_gradient_same_probes():
    """SLQ log determinant (Sec. 2) and the gradient of Eq. 1 with the
    quintic stencil equal the oracle's with identical probes (the GPU's
    pivots rebuilt in the oracle), as on the cubic path."""
    need_gpu()
    from oracle.mll import mll_grad_hutchinson_z
    from oracle.probes import preconditioned_probes
    from oracle.slq import slq_logdet_z
    from oracle.solve import QRPreconditioner, pivoted_cholesky
    p = Q(W.small2d(60, m=16, seed=11, nv=1e-2, ng=1e-2))
    op = gpu_op(p, "fp64")
    orc = oracle_op(p)
    pc = op.pivchol(20)
    _, piv = pc.export()
    Lo, _, _ = pivoted_cholesky(orc.kgrad_diag(), orc.kgrad_row, 20, pivots=piv)
    Pc = QRPreconditioner(Lo, orc.noise)
    P, seed = 12, 2024
    Z = preconditioned_probes(seed, Pc, P)
    ld, se = op.logdet(pc, probes=P, depth=12, seed=seed)
    est, se_o, _, _ = slq_logdet_z(orc.mvm, Pc, Z, depth=12, rtol=1e-15, maxit=12)
    assert abs(ld - est) <= 1e-10 * abs(est), (ld, est)
    P, seed = 16, 31
    mll, g = op.mll_grad(torch.tensor(p["y"], device="cuda"), pc, probes=P, seed=seed)
    Z = preconditioned_probes(seed, Pc, P)
    _, tr, go = mll_grad_hutchinson_z(orc, p["y"], Pc, Z, rtol=1e-12)
    assert np.allclose(g, go, rtol=1e-6, atol=1e-6 * np.abs(go).max()), (g, go)
    pc.close()
    op.close()
