"""Many independent D-SKI problems (uneven n and d) solved together.

persistent=True (the default): host threads build each problem's handle
and rank-r preconditioner on its own CUDA stream (ctypes releases the
interpreter lock, so the set-up kernels overlap), then ONE persistent launch
(dski_pcg_solve_batch) solves every system: a CTA per system, systems taken
from a device work queue, largest first.

persistent=False: each problem also solves on its own stream
(dski_pcg_solve), the GPU overlapping the per-problem kernels.

Argument marshalling only: every step runs in the CUDA library.
"""
import concurrent.futures as cf
import time

import torch

from . import DSKI, DskiError, solve_batch


def _setup(p, rank, prec, device):
    stream = torch.cuda.Stream(device=device)
    with torch.cuda.stream(stream):
        X = torch.as_tensor(p["X"], dtype=torch.float64).to(device, non_blocking=True)
        y = torch.as_tensor(p["y"], dtype=torch.float64).to(device, non_blocking=True)
        op = DSKI(X, p["m"], p["lo"], p["hi"], p["ell"], p["sf"], p["noise_value"],
                  p["noise_grad"], prec=prec, stream=stream)
        pc = op.pivchol(rank) if rank > 0 else None
    stream.synchronize()
    return op, pc, y


def solve_many(problems, rank=32, rtol=1e-6, maxit=20000, prec="fp64", workers=8,
               device="cuda", persistent=True, timings=None, cluster=0):
    """Solve K~_i x_i = y_i for every problem dict (X, y, m, lo, hi, ell, sf,
    noise_value, noise_grad).  Returns a list of dicts with x (CPU tensor),
    iters, relres, error (None, or the message / status of a solve that
    failed) and seconds: the problem's solve time inside the persistent
    launch (device clock), or its wall time on its stream.  timings (a
    dict, persistent mode): receives the wall seconds of the set-up
    ("setup_s") and of the persistent launch ("solve_s").  cluster: CTAs
    per system in the persistent launch (1, 2, 4 or 8; 0: the default)."""
    if persistent:
        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(max_workers=max(1, workers)) as ex:
            built = list(ex.map(lambda p: _setup(p, rank, prec, device), problems))
        ops = [b[0] for b in built]
        pcs = [b[1] for b in built]
        try:
            t1 = time.perf_counter()
            xs, its, rrs, status, secs = solve_batch(ops, pcs, [b[2] for b in built], rtol=rtol,
                                                     maxit=maxit, allow_failed=True,
                                                     cluster=cluster)
            if timings is not None:
                timings["setup_s"] = t1 - t0
                timings["solve_s"] = time.perf_counter() - t1
            out = []
            for x, it, rr, st, sec in zip(xs, its, rrs, status, secs):
                out.append({"x": x.to("cpu"), "iters": it, "relres": rr,
                            "error": None if st == "OK" else st, "seconds": sec})
            return out
        finally:
            for op, pc in zip(ops, pcs):
                if pc is not None:
                    pc.close()
                op.close()

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
