"""Failure handling on the GPU without a fault: a device-side wait that runs
out of its budget.

Every CTA of the tensor-core mode products waits on an mbarrier for its TMA
loads with a bounded number of polls.  dski_set_wait_budget(h, 0) makes that
first wait give up at once on a normal launch: the CTA records the device
error word, waits (with the full budget) for its own loads to land, frees its
tensor memory and returns.  The solver's next host check must return
DSKI_ERR_TIMEOUT, and the same handle must compute correct products
afterwards (the context stays usable).  Nothing here faults or hangs the GPU:
the loads always complete, only the wait for them is cut short.
"""
import numpy as np
import pytest

from synth import workloads as W
from tests._gpu_helpers import gpu_op, oracle_op, need_gpu, torch, check_mvm

pytestmark = pytest.mark.gpu


CASES = [
    # FP64_TC: the 64-node modes and the grid-form preconditioner's products
    # run on the digit-product kernel
    ("fp64_tc", lambda: dict(W.sine2d(), m=(64, 64))),
    # MIXED: 32-node modes take the clustered split contraction; noise 1e-2,
    # which the FP32 operator resolves
    ("mixed_3xtf32", lambda: dict(W.small2d(300, m=16, seed=21, nv=1e-2, ng=1e-2), m=(32, 32))),
]


@pytest.mark.parametrize("prec,make", CASES, ids=["fp64_tc-digit-products",
                                                   "mixed-split-contraction"])
def test_wait_that_runs_out_returns_timeout_and_handle_recovers(prec, make):
    need_gpu()
    from paper_1810_12283_gb300 import DskiError
    p = make()
    op = gpu_op(p, prec)
    orc = oracle_op(p)
    pc = op.pivchol(20)
    b = torch.tensor(p["y"], device="cuda")
    op.set_wait_budget(0)
    with pytest.raises(DskiError) as e:
        op.solve(b, pc, rtol=1e-8, maxit=64)
    assert e.value.status == "TIMEOUT"
    # default budget again: the same handle gives correct products and solves
    op.set_wait_budget(-1)
    v = np.random.default_rng(3).normal(size=orc.N)
    got = op.mvm(torch.tensor(v, device="cuda")).double().cpu().numpy()
    vin = v if prec == "fp64_tc" else v.astype(np.float32).astype(np.float64)
    check_mvm(orc, vin, got, prec)
    x, it, rr = op.solve(b, pc, rtol=1e-6, maxit=20000)
    assert rr[0] <= 1e-6
    A = orc.dense()
    assert np.linalg.norm(p["y"] - A @ x.cpu().numpy()) / np.linalg.norm(p["y"]) <= 1.5e-6
    pc.close()
    op.close()
