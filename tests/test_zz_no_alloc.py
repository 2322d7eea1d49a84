"""dski_mvm_noalloc, the MVM entry point for callers that cannot allocate
device memory (their memory belongs to a pool allocator, or cudaMalloc's
implicit synchronisation is not allowed where they run).  It keeps its
temporaries in a fixed device array, so it must give the same product as
dski_mvm, call after call, refuse sizes that do not fit that array, and
allocate nothing even on a fresh handle.

This file is collected last on purpose: a failure here stops a run only after
every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

from synth import workloads as W
from tests._gpu_helpers import gpu_op, need_gpu, oracle_op, rel, torch, mvm_tolerance

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed_3xtf32": 1e-6}


def _call(lib, op, fn, V, out=None):
    out = torch.empty_like(V) if out is None else out
    rc = getattr(lib, fn)(op.h, C.c_void_p(V.data_ptr()), C.c_void_p(out.data_ptr()), V.shape[0])
    return rc, out


def _quintic(p):
    q = dict(p)
    q["interp"] = "quintic"
    return q


@pytest.mark.parametrize("prec", ["fp64", "mixed_3xtf32"])
def test_noalloc_matches_mvm_on_consecutive_calls(prec):
    need_gpu()
    from paper_1810_12283_gb300 import _lib
    lib = _lib.load()
    cases = [(lambda: W.small3d(300, m=11, seed=4), 3), (lambda: W.sine2d(), 2)]
    if prec == "fp64":
        # the quintic stencil's per-point intermediate (2 S and 2 S^2 doubles, S = 6)
        cases += [(lambda: _quintic(W.small2d(400, m=21, seed=5)), 3),
                  (lambda: _quintic(W.small3d(200, m=14, seed=6)), 2)]
    for make, s in cases:
        op = gpu_op(make(), prec)
        g = torch.Generator(device="cuda")
        g.manual_seed(7)
        # two calls in a row with different inputs: the second must not see the first
        for _ in range(2):
            V = torch.randn(s, op.N, device="cuda", dtype=op.dtype, generator=g)
            rc_ref, ref = _call(lib, op, "dski_mvm", V)
            rc, got = _call(lib, op, "dski_mvm_noalloc", V)
            assert rc_ref == 0 and rc == 0, lib.dski_last_error()
            torch.cuda.synchronize()
            for q in range(s):
                assert rel(got[q].double().cpu().numpy(), ref[q].double().cpu().numpy()) <= TOL[prec]
        op.close()


def _terrain_like(n, seed):
    # a 256^2 grid (the terrain grid) with few points: in the MIXED modes its
    # mode products take the clustered split contraction, whose partials for
    # s = 4 (8 MB) are far above the driver's allocation granularity
    p = W.terrain2d(n=n, seed=seed, features=64)
    return p


def test_noalloc_fresh_mixed_handle_allocates_nothing():
    need_gpu()
    from paper_1810_12283_gb300 import _lib
    lib = _lib.load()
    s = 4
    # warm-up on another handle: loads the kernels (lazy module loading takes
    # device memory at a kernel's first launch) and looks up the array
    warm = gpu_op(_terrain_like(2000, 11), "mixed_3xtf32")
    Vw = torch.randn(s, warm.N, device="cuda", dtype=torch.float32)
    rc, _ = _call(lib, warm, "dski_mvm_noalloc", Vw)
    assert rc == 0, lib.dski_last_error()
    torch.cuda.synchronize()
    warm.close()

    p = _terrain_like(2000, 12)
    op = gpu_op(p, "mixed_3xtf32")        # fresh: dski_mvm has never run on it
    rng = np.random.default_rng(3)
    Vh = rng.normal(size=(s, op.N))
    V = torch.tensor(Vh, device="cuda", dtype=torch.float32)
    out = torch.empty_like(V)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        rc, _ = _call(lib, op, "dski_mvm_noalloc", V, out)
        assert rc == 0, lib.dski_last_error()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
    got = out.double().cpu().numpy()
    # against the oracle, at the mixed-mode tolerance derived from the arithmetic
    orc = oracle_op(p)
    Vr = V.double().cpu().numpy()     # the FP32 input the GPU saw
    for q in range(s):
        tol = mvm_tolerance(orc, Vr[q], "mixed_3xtf32")
        assert rel(got[q], orc.mvm(Vr[q])) <= tol
    # and against dski_mvm on the same handle
    rc_ref, ref = _call(lib, op, "dski_mvm", V)
    assert rc_ref == 0
    torch.cuda.synchronize()
    for q in range(s):
        assert rel(got[q], ref[q].double().cpu().numpy()) <= TOL["mixed_3xtf32"]
    op.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    need_gpu()
    from paper_1810_12283_gb300 import _lib
    lib = _lib.load()
    op = gpu_op(W.small2d(2000, m=16, seed=1), "fp64")
    s = 400   # 2 N s + 2 M s doubles = 41 MB > 32 MiB
    V = torch.zeros(s, op.N, device="cuda", dtype=torch.float64)
    rc, _ = _call(lib, op, "dski_mvm_noalloc", V)
    assert rc == -1
    assert b"fixed limit" in lib.dski_last_error()
    # a fitting call still works afterwards
    V = torch.randn(2, op.N, device="cuda", dtype=torch.float64)
    rc_ref, ref = _call(lib, op, "dski_mvm", V)
    rc, got = _call(lib, op, "dski_mvm_noalloc", V)
    assert rc == 0 and rc_ref == 0
    assert rel(got.cpu().numpy(), ref.cpu().numpy()) <= TOL["fp64"]
    op.close()
