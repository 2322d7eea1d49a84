"""Many independent D-SKI problems (uneven n and d) solved concurrently.

Each problem gets its own D-SKI handle on its own CUDA stream; host threads
drive the C-ABI calls (ctypes releases the interpreter lock), so the GPU
overlaps the small per-problem kernels.  Argument marshalling only: every
step runs in the CUDA library.
"""
import concurrent.futures as cf
import time

import torch

from . import DSKI, DskiError


def solve_many(problems, rank=32, rtol=1e-6, maxit=20000, prec="fp64", workers=8,
               device="cuda"):
    """Solve K~_i x_i = y_i for every problem dict (X, y, m, lo, hi, ell, sf,
    noise_value, noise_grad).  Returns a list of dicts with x (CPU tensor),
    iters, relres, error (None, or the message of a solve that failed, whose
    x is None) and the problem's wall time."""

    def one(p):
        stream = torch.cuda.Stream(device=device)
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            X = torch.as_tensor(p["X"], dtype=torch.float64).to(device, non_blocking=True)
            y = torch.as_tensor(p["y"], dtype=torch.float64).to(device, non_blocking=True)
            op = DSKI(X, p["m"], p["lo"], p["hi"], p["ell"], p["sf"], p["noise_value"],
                      p["noise_grad"], prec=prec, stream=stream)
            pc = op.pivchol(rank)
            err = None
            try:
                x, it, rr = op.solve(y, pc, rtol=rtol, maxit=maxit, allow_not_converged=True)
                xh = x.to("cpu")
            except DskiError as e:   # e.g. a breakdown of a mode the problem defeats
                err, xh, it, rr = str(e), None, [0], [float("nan")]
            finally:
                pc.close()
                op.close()
        stream.synchronize()
        return {"x": xh, "iters": it[0], "relres": rr[0], "error": err,
                "seconds": time.perf_counter() - t0}

    with cf.ThreadPoolExecutor(max_workers=max(1, workers)) as ex:
        return list(ex.map(one, problems))
