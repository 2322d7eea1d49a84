"""Many uneven problems at once (the multi-instance pattern).

The stream-concurrent driver gives each problem exactly the solution a lone
solve gives (the kernels are deterministic).  The persistent launch
(dski_pcg_solve_batch, a CTA per system) runs the same PCG in its own
kernel.  Every solution meets the tolerance by its FP64 true residual and
satisfies the oracle's system: ||y - K~_oracle x|| / ||y|| within 1.5x the
tolerance."""
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
    res = solve_many(probs, rank=16, rtol=1e-6, maxit=20000, workers=3, persistent=False)
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


# ---- the persistent launch (dski_pcg_solve_batch) -------------------------

def _persistent_cases():
    from tests._gpu_helpers import problem_1d
    probs = _small_instances(7)
    q = dict(W.small2d(300, m=21, seed=5))   # quintic stencil, no preconditioner
    q["interp"] = "quintic"
    probs.insert(3, problem_1d(300, m=40, seed=2))   # d = 1
    probs.append(q)
    return probs


@pytest.mark.parametrize("cluster", [1, 2, 4, 8])
def test_persistent_batch_meets_the_oracle_system(cluster):
    """Every system of one persistent launch -- 1-D, 2-D and 3-D, cubic and
    quintic, with and without a preconditioner -- reaches the FP64 tolerance
    by its own true residual and satisfies the oracle's system, whether one
    CTA or a cluster of 2, 4 or 8 CTAs solves each system."""
    need_gpu()
    from paper_1810_12283_gb300 import solve_batch
    probs = _persistent_cases()
    ops = [gpu_op(p, "fp64") for p in probs]
    pcs = [op.pivchol(16) if i < len(probs) - 1 else None for i, op in enumerate(ops)]
    bs = [torch.tensor(p["y"], device="cuda") for p in probs]
    xs, its, rrs, status, secs = solve_batch(ops, pcs, bs, rtol=1e-8, maxit=50000,
                                             cluster=cluster)
    assert status == ["OK"] * len(probs)
    for p, x, it, rr, sec in zip(probs, xs, its, rrs, secs):
        assert 0 < it < 50000 and rr <= 1e-8 and sec > 0
        orc = oracle_op(p)
        res = np.linalg.norm(p["y"] - orc.mvm(x.cpu().numpy())) / np.linalg.norm(p["y"])
        assert res <= 1.5e-8, (p.get("name"), res)
    # the same systems solved one by one (dski_pcg_solve) need about as many
    # iterations: both run the same PCG on the same operator
    for i in (0, 1):
        x1, it1, rr1 = ops[i].solve(bs[i], pcs[i], rtol=1e-8, maxit=50000)
        assert abs(it1[0] - its[i]) <= max(5, 0.1 * it1[0]), (it1[0], its[i])
    for pc in pcs:
        if pc is not None:
            pc.close()
    for op in ops:
        op.close()


def test_persistent_batch_edge_cases():
    """A zero right-hand side gives x = 0; a warm start at the solution
    needs no iteration; maxit = 3 reports NOT_CONVERGED with every output
    filled; unsupported handles are refused before anything runs."""
    need_gpu()
    from paper_1810_12283_gb300 import DskiError, solve_batch
    probs = _small_instances(3)
    ops = [gpu_op(p, "fp64") for p in probs]
    pcs = [op.pivchol(8) for op in ops]
    bs = [torch.tensor(p["y"], device="cuda") for p in probs]
    bs0 = [torch.zeros_like(bs[0])] + bs[1:]
    xs, its, rrs, status, _ = solve_batch(ops, pcs, bs0, rtol=1e-8, maxit=50000)
    assert status == ["OK"] * 3 and its[0] == 0 and rrs[0] == 0.0
    assert float(xs[0].abs().max()) == 0.0
    # warm start from the converged solutions (the scatter's shared-memory
    # atomics add in no fixed order, so the recomputed residual may differ
    # from the first in its last bits)
    xs2, its2, rrs2, status2, _ = solve_batch(ops, pcs, bs, rtol=1e-6, maxit=50000, x0s=xs)
    assert status2 == ["OK"] * 3
    assert its2[0] > 0 and all(i == 0 for i in its2[1:]) and max(rrs2[1:]) <= 1.01e-8
    # too few iterations
    xs3, its3, rrs3, status3, _ = solve_batch(ops, pcs, bs, rtol=1e-12, maxit=3,
                                              allow_failed=True, cluster=2)
    assert status3 == ["NOT_CONVERGED"] * 3 and its3 == [3, 3, 3]
    assert all(np.isfinite(r) and r > 1e-12 for r in rrs3)
    assert all(bool(torch.isfinite(x).all()) for x in xs3)
    with pytest.raises(DskiError) as e:
        solve_batch(ops, pcs, bs, rtol=1e-12, maxit=3)
    assert e.value.status == "NOT_CONVERGED"
    # a MIXED handle, and a grid too large for one CTA's shared memory
    mixed = gpu_op(probs[1], "mixed_3xtf32")
    with pytest.raises(DskiError) as e:
        solve_batch([mixed], [None], [bs[1]], rtol=1e-6)
    assert e.value.status == "ARG"
    mixed.close()
    big = W.small3d(200, m=40, seed=3)
    opb = gpu_op(big, "fp64")
    with pytest.raises(DskiError) as e:
        solve_batch([opb], [None], [torch.tensor(big["y"], device="cuda")], rtol=1e-6)
    assert e.value.status == "ARG" and "shared" in str(e.value)
    opb.close()
    with pytest.raises(DskiError) as e:
        solve_batch(ops, pcs, bs, rtol=1e-6, cluster=3)
    assert e.value.status == "ARG"
    for pc in pcs:
        pc.close()
    for op in ops:
        op.close()
