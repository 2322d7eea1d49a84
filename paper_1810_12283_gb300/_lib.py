"""ctypes declarations of the C ABI in ``include/dski.h``.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Loading fails loudly when ``libdski.so`` is missing (there is no
CPU fallback).
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdski.so")

DSKI_OK = 0
STATUS = {0: "OK", -1: "ARG", -2: "OUT_OF_GRID", -3: "CUDA", -4: "NOT_CONVERGED",
          -5: "BREAKDOWN", -6: "TIMEOUT", -7: "ALLOC"}
PREC = {"fp64": 0, "mixed_3xtf32": 1, "mixed_tf32": 2, "fp64_tc": 3}
INTERP = {"cubic": 0, "quintic": 1}
KUU = {"dense": 0, "fft": 1}

# every extern "C" symbol include/dski.h declares
EXPORTS = ["dski_create", "dski_set_hypers", "dski_mvm", "pivchol_build", "dski_pcg_solve",
           "dski_logdet_slq", "dski_mll_grad", "dski_destroy", "pivchol_destroy",
           "dski_last_error", "dski_profile", "dski_launch_count", "pivchol_export",
           "pivchol_logdet", "dski_mvm_noalloc", "dski_predict", "dski_predict_var_cv",
           "dski_mll_grad_tol", "dski_set_wait_budget", "dski_pcg_solve_batch"]
NSTAGES = 8
STAGES = ["permute", "scatter", "kron", "gather", "precond", "pcg_vec", "pivchol", "lanczos"]


class DskiParams(C.Structure):
    _fields_ = [("n", C.c_int), ("d", C.c_int),
                ("grid_m", C.POINTER(C.c_int)),
                ("grid_lo", C.POINTER(C.c_double)),
                ("grid_hi", C.POINTER(C.c_double)),
                ("lengthscale", C.POINTER(C.c_double)),
                ("outputscale", C.c_double),
                ("noise_value", C.c_double), ("noise_grad", C.c_double),
                ("prec", C.c_int), ("interp", C.c_int), ("kuu", C.c_int)]


class DskiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


_lib = None


def load(path=LIB_PATH):
    """Load (once) and declare the library."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libdski.so not built ({path}); run paper_1810_12283_gb300.build.build()")
    lib = C.CDLL(path)
    vp, ip, dp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)
    lib.dski_create.argtypes = [C.POINTER(vp), C.POINTER(DskiParams), vp, vp]
    lib.dski_set_hypers.argtypes = [vp, dp, C.c_double, C.c_double, C.c_double]
    lib.dski_mvm.argtypes = [vp, vp, vp, C.c_int]
    lib.dski_mvm_noalloc.argtypes = [vp, vp, vp, C.c_int]
    lib.pivchol_build.argtypes = [vp, C.c_int, C.POINTER(vp), ip]
    lib.dski_pcg_solve.argtypes = [vp, vp, vp, vp, C.c_int, C.c_double, C.c_int, ip, dp]
    lib.dski_logdet_slq.argtypes = [vp, vp, C.c_int, C.c_int, C.c_uint64, dp, dp]
    lib.dski_mll_grad.argtypes = [vp, vp, vp, C.c_int, C.c_uint64, dp, dp]
    lib.dski_mll_grad_tol.argtypes = [vp, vp, vp, C.c_int, C.c_uint64, C.c_double, C.c_int,
                                      dp, dp]
    lib.dski_set_wait_budget.argtypes = [vp, C.c_int]
    lib.dski_pcg_solve_batch.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                                         C.POINTER(vp), C.c_double, C.c_int, C.c_int, ip, dp, ip,
                                         dp]
    lib.dski_predict.argtypes = [vp, vp, vp, vp, C.c_int, C.c_int, vp, vp]
    lib.dski_predict_var_cv.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_uint64, C.c_double,
                                        C.c_int, vp]
    lib.dski_destroy.argtypes = [vp]
    lib.dski_destroy.restype = None
    lib.pivchol_destroy.argtypes = [vp]
    lib.pivchol_destroy.restype = None
    lib.dski_last_error.restype = C.c_char_p
    lib.dski_profile.argtypes = [vp, C.c_int, dp, C.POINTER(C.c_longlong),
                                 C.POINTER(C.c_longlong), ip]
    lib.dski_launch_count.argtypes = []
    lib.dski_launch_count.restype = C.c_longlong
    lib.pivchol_export.argtypes = [vp, vp, ip]
    lib.pivchol_logdet.argtypes = [vp]
    lib.pivchol_logdet.restype = C.c_double
    for name in EXPORTS:
        if name not in ("dski_destroy", "pivchol_destroy", "dski_last_error",
                        "dski_launch_count", "pivchol_logdet"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def check(rc, allow=()):
    if rc != DSKI_OK and rc not in allow:
        raise DskiError(rc, load().dski_last_error().decode(errors="replace"))
    return rc
