"""Many uneven problems at once (the multi-instance pattern): the
stream-concurrent driver gives each problem exactly the solution a lone
solve gives (the kernels are deterministic), meets the tolerance, and each
solution satisfies the oracle's system: ||y - K~_oracle x|| / ||y|| within
1.5x the tolerance."""
import numpy as np
import pytest

from synth import workloads as W
from tests._gpu_helpers import gpu_op, need_gpu, oracle_op, torch

pytestmark = pytest.mark.gpu


def _small_instances(k):
    out = []
    for i in range(k):
        p = W.multi_instance(i)
        n = min(p["X"].shape[0], 400)
        out.append(W.subsample(p, n, seed=i))
    return out


def test_solve_many_matches_single_solves():
    need_gpu()
    from paper_1810_12283_gb300.batch import solve_many
    probs = _small_instances(6)
    assert {q["X"].shape[1] for q in probs} == {2, 3}
    res = solve_many(probs, rank=16, rtol=1e-6, maxit=20000, workers=3)
    for p, r in zip(probs, res):
        op = gpu_op(p, "fp64")
        pc = op.pivchol(16)
        x, it, rr = op.solve(torch.tensor(p["y"], device="cuda"), pc, rtol=1e-6, maxit=20000)
        assert r["relres"] <= 1e-6 and it[0] == r["iters"]
        assert np.array_equal(r["x"].numpy(), x.cpu().numpy())
        orc = oracle_op(p)
        res = np.linalg.norm(p["y"] - orc.mvm(r["x"].numpy())) / np.linalg.norm(p["y"])
        assert res <= 1.5e-6, res
        pc.close()
        op.close()
