"""dski_mvm_noalloc, the MVM entry point for callers that cannot allocate
device memory (their memory belongs to a pool allocator, or cudaMalloc's
implicit synchronisation is not allowed where they run).  It keeps its
temporaries in a fixed device array, so it must give the same product as
dski_mvm, call after call, and refuse sizes that do not fit that array.

This file is collected last on purpose: a failure here stops a run only after
every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

from synth import workloads as W
from tests._gpu_helpers import gpu_op, need_gpu, rel, torch

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed_3xtf32": 1e-6}


def _call(lib, op, fn, V):
    out = torch.empty_like(V)
    rc = getattr(lib, fn)(op.h, C.c_void_p(V.data_ptr()), C.c_void_p(out.data_ptr()), V.shape[0])
    return rc, out


@pytest.mark.parametrize("prec", ["fp64", "mixed_3xtf32"])
def test_noalloc_matches_mvm_on_consecutive_calls(prec):
    need_gpu()
    from paper_1810_12283_gb300 import _lib
    lib = _lib.load()
    for make, s in ((lambda: W.small3d(300, m=11, seed=4), 3), (lambda: W.sine2d(), 2)):
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
