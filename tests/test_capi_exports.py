"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads,
and exports every symbol that include/dski.h declares."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "dski.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b((?:dski|pivchol)_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("dski_create", "dski_mvm", "dski_pcg_solve", "dski_logdet_slq", "pivchol_build"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    from paper_1810_12283_gb300 import build, _lib
    try:
        path = build.build()
    except RuntimeError as e:   # no nvcc on this machine
        pytest.skip(str(e))
    lib = _lib.load(path)
    for s in declared_symbols():
        assert hasattr(lib, s), s
    assert set(declared_symbols()) <= set(_lib.EXPORTS) | set(declared_symbols())
    assert sorted(_lib.EXPORTS) == declared_symbols()


def test_last_error_empty_initially():
    from paper_1810_12283_gb300 import build, _lib
    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    assert isinstance(_lib.load().dski_last_error(), bytes)


def _lib_or_skip():
    from paper_1810_12283_gb300 import build, _lib
    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    return _lib, _lib.load()


def test_invalid_arguments_are_rejected_before_any_device_work():
    """dski_create validates the problem statement (Sec. 2 / Sec. 3.1 sizes,
    App. A hyperparameters) on the host and returns DSKI_ERR_ARG with a
    message; the other calls reject NULL handles the same way."""
    import ctypes as C
    _lib, lib = _lib_or_skip()
    m = (C.c_int * 2)(16, 16)
    lo = (C.c_double * 2)(0.0, 0.0)
    hi = (C.c_double * 2)(1.0, 1.0)
    ell = (C.c_double * 2)(0.2, 0.2)
    dummy = C.c_void_p(1)   # never dereferenced: validation fails first

    def create(**kw):
        f = dict(n=10, d=2, grid_m=m, grid_lo=lo, grid_hi=hi, lengthscale=ell, outputscale=1.0,
                 noise_value=1e-3, noise_grad=1e-3, prec=0, interp=0, kuu=0)
        f.update(kw)
        p = _lib.DskiParams(f["n"], f["d"], f["grid_m"], f["grid_lo"], f["grid_hi"],
                            f["lengthscale"], f["outputscale"], f["noise_value"],
                            f["noise_grad"], f["prec"], f["interp"], f["kuu"])
        h = C.c_void_p()
        rc = lib.dski_create(C.byref(h), C.byref(p), dummy, None)
        return rc, lib.dski_last_error().decode()

    assert create(n=0) == (-1, "dski_create: n must be >= 1 (got 0)")
    assert create(d=4)[0] == -1
    assert create(prec=9)[0] == -1
    assert create(outputscale=0.0)[0] == -1
    assert create(noise_grad=-1.0)[0] == -1
    assert create(grid_m=(C.c_int * 2)(3, 16))[0] == -1
    assert create(grid_hi=(C.c_double * 2)(0.0, 1.0))[0] == -1
    assert create(lengthscale=(C.c_double * 2)(0.2, float("nan")))[0] == -1
    assert create(prec=3, grid_m=(C.c_int * 2)(20, 16))[0] == -1   # FP64_TC needs m % 8 == 0
    # interpolation scheme and K_UU product (Sec. 3.1)
    assert create(interp=2)[0] == -1
    assert create(interp=1, grid_m=(C.c_int * 2)(5, 16)) == \
        (-1, "dski_create: grid_m[0] must be in 6..1027 (got 5)")   # quintic: 6 nodes
    assert create(kuu=2)[0] == -1
    assert create(kuu=1, prec=1) == \
        (-1, "dski_create: the FFT K_UU product needs FP64 vectors (FP64 or FP64_TC)")
    assert lib.dski_mvm(None, dummy, dummy, 1) == -1
    assert lib.dski_pcg_solve(None, None, dummy, dummy, 1, 1e-8, 10, None, None) == -1
    assert lib.dski_mvm_noalloc(None, dummy, dummy, 1) == -1
    out = C.c_void_p(7)
    got = C.c_int()
    assert lib.pivchol_build(None, 10, C.byref(out), C.byref(got)) == -1
    assert out.value is None
