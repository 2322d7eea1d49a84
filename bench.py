"""Benchmark of the D-SKI hot path on one GB300 (or N independent replicas).

Workload: the terrain stand-in -- n = 100,000 points uniform in [0,1]^2 with
values and gradients of a 512-feature random Fourier field (N = 300,000
rows), SE length scale 0.05, noise 1e-3, 256 x 256 grid over
[-0.05, 1.05]^2, pivoted-Cholesky rank 100, PCG to relative residual 1e-8.
Inputs are synthetic and seeded (``synth.workloads.terrain2d``).

A step is one pass of the whole hot path: build the D-SKI operator for the
resident points (geometry, sort, factors), the rank-100 pivoted Cholesky and
its QR-form preconditioner, and the PCG solve K~ x = y to 1e-8 (true FP64
residual).  The headline mode is FP64_TC: the Kronecker mode products run on
the BF16 tensor cores as exact digit-pair products (FP64-accurate), the true
residuals of the restarts use the FP64 units.  The plain FP64 mode runs the
same step to the same tolerance beside it; MIXED_3XTF32 runs it with an
iteration cap of min(1.5x the headline count, 30000) and reports the residual
it reaches (its FP32 operator error exceeds the noise variance here).  Each
mode's MVM throughput is timed separately.  The L2 is flushed (a 256 MiB
write) before every timed step, outside the timed events.

Printed: one JSON line (rank 0).  ``--impl reference`` times the plain FP64
CPU oracle instead (the reference arm of this project).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# the headline metric (PCG solve seconds and D-SKI MVM HBM GB/s, mixed
# vs FP64, on the terrain workload at relative residual 1e-8); `value` is the
# solve time of the headline mode, the other modes sit under "compare"
METRIC = "PCG solve s & D-SKI MVM HBM GB/s: mixed vs FP64, same GB300, rel res 1e-8"
UNIT = "s"
RANK = 100
PROF_ITERS = 3000   # PCG iterations of the profiled (untimed) step
RTOL = 1e-8


def workload_name(n, interp="cubic", kuu="dense"):
    tail = ("" if interp == "cubic" else f" interp={interp}") + ("" if kuu == "dense" else f" kuu={kuu}")
    return f"terrain2d n={n} d=2 N={3 * n} grid=256x256 rank={RANK} rtol={RTOL:g}{tail}"


def stencil_nodes(interp):
    """Nodes per dimension of the interpolation stencil."""
    return 6 if interp == "quintic" else 4


def geometry_bytes(d, elem):
    """Per-point geometry the scatter and gather need: the int32 cell id and
    d cell fractions in the vector precision (g = 4 + 4 d bytes with FP32
    vectors, 4 + 8 d with FP64)."""
    return 4 + elem * d


def weight_table_bytes(d, elem, S=4):
    """Per-point bytes of the precomputed stencil weight tables the kernels
    read instead of recomputing the weights from the fractions (S weights
    and S derivative weights per dimension): traffic beyond the algorithmic
    model, reported separately."""
    return elem * 2 * S * d


def mvm_bytes(n, d, s, elem):
    """Algorithmic HBM bytes of one MVM: v read by the scatter and by the
    noise term, out written (3 N s elements), the per-point geometry read by
    scatter and gather (2 n g).  The grid stays in L2."""
    N = n * (d + 1)
    return 3 * N * s * elem + 2 * n * geometry_bytes(d, elem)


def scatter_bytes(n, d, M, s, elem):
    """Algorithmic bytes of one scatter: v read (N s elements), the geometry
    read (n g), the grid written (M s elements)."""
    N = n * (d + 1)
    return N * s * elem + n * geometry_bytes(d, elem) + M * s * elem


def gather_bytes(n, d, M, s, elem):
    """Algorithmic bytes of one gather with the noise term: the grid (M s)
    and v (N s) read, the geometry read (n g), out (N s) written."""
    N = n * (d + 1)
    return M * s * elem + 2 * N * s * elem + n * geometry_bytes(d, elem)


OZ_PAIRS = 36   # digit pairs (a, b), a + b < 8, of the FP64_TC mode product


def scatter_flops(n, d, S=4):
    """Algorithmic FP64 flops of one d = 2 scatter in its sum-factorised form,
    per point: 3 scalings, S c_a = w_a v0 + w'_a v1 (3 flops each), S e_a =
    w_a v2, then S^2 stencil nodes x (w1_b c_a + w1'_b e_a) (2 FMAs)."""
    assert d == 2
    return n * (3 + S * 3 + S + S * S * 4)


def batch_iter_flops(n, d, M, msum, rank, S=4):
    """FP64 flops of one PCG iteration of the persistent batched solver for
    one system (n points in d dimensions, M grid nodes, sum of m_k msum, a
    rank-`rank` QR-form preconditioner), counting an FMA as 2 flops, in the
    sum-factorised form the kernel evaluates:
      scatter per point   d = 2: S (3 + 1) + S^2 (3 + 1 atomic add)
                          d = 3: S (3 + 1 + 1) + S^2 (3 + 1) + S^3 (3 + 1)
      gather per point    d = 2: 4 S^2 + 6 S;  d = 3: 4 S^3 + 6 S^2 + 8 S
      per row             noise and p^T q 4, p update 2, x and r updates 4,
                          ||r||^2 2, D^-1/2 r 1, c = Q1^T y 2 rank,
                          z 2 + 2 rank, r^T z 2
      mode products       2 M sum_k m_k."""
    if d == 1:
        scat, gath = S * 4, S * 4
    elif d == 2:
        scat, gath = S * 4 + S * S * 4, 4 * S * S + 6 * S
    elif d == 3:
        scat, gath = S * 5 + S * S * 4 + S ** 3 * 4, 4 * S ** 3 + 6 * S * S + 8 * S
    else:
        raise ValueError("d must be 1, 2 or 3")
    N = n * (d + 1)
    return n * (scat + gath) + 2 * M * msum + N * (17 + 4 * rank)


def measure_peaks(dev):
    """Dense-GEMM rates of this GPU measured in the run (CUDA events, best of
    3 after a warm-up): FP64 (cuBLAS DGEMM, 8192^3) and TF32 (cuBLAS FP32
    GEMM on the TF32 tensor cores, 8192^3), in TFLOP/s."""
    import torch
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    for name, dt, tf32, nn in (("fp64_tflops", torch.float64, False, 8192),
                               ("tf32_tflops", torch.float32, True, 8192)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(nn, nn, device=dev, dtype=dt)
        b = torch.randn(nn, nn, device=dev, dtype=dt)
        c = a @ b
        best = 1e30
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        out[name] = 2.0 * nn ** 3 / best / 1e12
        del a, b, c
    torch.backends.cuda.matmul.allow_tf32 = prev
    torch.cuda.empty_cache()
    return out


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch.distributed as dist
    dist.init_process_group(os.environ.get("DSKI_BENCH_BACKEND", "nccl"))
    return dist.get_rank(), dist.get_world_size(), dist


def reduce_max(dist, value, device):
    """Max over ranks of a host float (identity on one process)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# the FP64 PCG iteration count of the terrain solve to 1e-8 measured on
# GB300 (the FP64 mode's "compare" entry of the bench line); the reference
# arm, which runs no GPU code, scales its per-iteration oracle time to it
FP64_TERRAIN_ITERS = 120158


def oracle_operator(p):
    """The oracle's D-SKI operator and rank-100 preconditioner for problem p,
    and the seconds the set-up took."""
    from oracle.dski import DSKI as ODSKI, Grid
    from oracle.solve import QRPreconditioner, pivoted_cholesky
    t0 = time.perf_counter()
    op = ODSKI(p["X"], Grid(p["m"], p["lo"], p["hi"], p.get("interp", "cubic")), p["ell"],
               p["sf"], p["noise_value"], p["noise_grad"])
    L, _, _ = pivoted_cholesky(op.kgrad_diag(), op.kgrad_row, RANK)
    Pc = QRPreconditioner(L, op.noise)
    return op, Pc, time.perf_counter() - t0


def cpu_baseline(p, iters_scaled_to, iters_source, budget_s=12.0, built=None):
    """The FP64 oracle on the host cores: operator build, rank-100 pivoted
    Cholesky and QR preconditioner (timed whole), then PCG iterations timed
    on a bounded sample and scaled to `iters_scaled_to` iterations -- an
    extrapolation, labelled as such.  `built`: (op, Pc, setup seconds) from
    oracle_operator, reused."""
    from oracle.solve import pcg
    op, Pc, t_setup = built if built is not None else oracle_operator(p)
    k = 5
    while True:
        t0 = time.perf_counter()
        pcg(op.mvm, p["y"], Pc.solve, rtol=0.0, maxit=k)
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or k >= 4000:
            break
        k = int(k * max(2.0, min(8.0, budget_s / 4 / max(dt, 1e-3))))
    per_it = dt / k
    est = t_setup + per_it * iters_scaled_to
    return {"value": est, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
            "extrapolated": True, "iters_timed": k, "iters_scaled_to": int(iters_scaled_to),
            "iters_source": iters_source, "setup_s": t_setup, "s_per_iter": per_it,
            "sample": (f"oracle setup (operator, rank-{RANK} pivoted Cholesky, QR) timed whole "
                       f"({t_setup:.1f} s); {k} oracle PCG iterations timed ({dt:.1f} s, "
                       f"{per_it * 1e3:.1f} ms each), extrapolated to {int(iters_scaled_to)} "
                       f"iterations ({iters_source})")}


SUB_N, SUB_SEED, SUB_PROBES, SUB_DEPTH = 1000, 9, 8, 12
SUB_RTOL = 1e-8   # FP64 PCG attains ~2-4e-9 on this subsample (measured)


def gpu_subsample_run(DSKI, p, prec, dev):
    """The GPU's solve, SLQ log determinant and Eq. 1 gradient on a seeded
    1000-point subsample of the workload (same grid and hyperparameters),
    for the oracle check.  Returns host values and the GPU's pivots."""
    import torch
    from synth import workloads as W
    q = W.subsample(p, SUB_N, seed=SUB_SEED)
    op = DSKI(torch.tensor(q["X"], device=dev), q["m"], q["lo"], q["hi"], q["ell"], q["sf"],
              q["noise_value"], q["noise_grad"], prec=prec, interp=p["interp"], kuu=p["kuu"])
    pc = op.pivchol(RANK)
    _, piv = pc.export()
    y = torch.tensor(q["y"], device=dev)
    out = {"prec": prec, "q": q, "piv": piv, "rank": pc.rank}
    try:
        x, it, rr = op.solve(y, pc, rtol=SUB_RTOL, maxit=200000, allow_not_converged=True)
        out.update(x=x.cpu().numpy(), iters=it[0], relres=rr[0])
    except Exception as e:   # noqa: BLE001 -- reported
        out["solve_error"] = str(e)
    try:
        out["logdet"], out["logdet_se"] = op.logdet(pc, probes=SUB_PROBES, depth=SUB_DEPTH,
                                                    seed=777)
    except Exception as e:   # noqa: BLE001
        out["logdet_error"] = str(e)
    try:
        out["mll"], out["grad"] = op.mll_grad(y, pc, probes=SUB_PROBES, seed=31, rtol=SUB_RTOL,
                                              maxit=200000)
    except Exception as e:   # noqa: BLE001
        out["grad_error"] = str(e)
    pc.close()
    op.close()
    return out


def oracle_check(p, built, xs, subs):
    """Errors of the GPU's results against the FP64 oracle (untimed).
    xs: {mode: x} full-size solutions (host, block order):
      relres_oracle = ||y - K~_oracle x|| / ||y||.
    subs: gpu_subsample_run results: the subsample's solve against the dense
    direct solve, the SLQ log determinant against the oracle's with the same
    probes (and the exact dense log determinant, in GPU standard errors),
    the gradient of Eq. 1 against the oracle's same-probe estimator (solves
    from the dense Cholesky factor) and the exact dense gradient."""
    import numpy as np
    from oracle.dski import DSKI as ODSKI, Grid
    from oracle.mll import mll_grad_dense, mll_grad_hutchinson_direct
    from oracle.probes import preconditioned_probes
    from oracle.slq import slq_logdet_z
    from oracle.solve import QRPreconditioner, chol_logdet, chol_solve, pivoted_cholesky
    from oracle.mll import _dense_matrix
    op = built[0]
    y = p["y"]
    out = {"full": {}}
    ny = float(np.linalg.norm(y))
    for mode, x in xs.items():
        out["full"][mode] = {"relres_oracle": float(np.linalg.norm(y - op.mvm(x)) / ny)}
    for sub in subs:
        q = sub["q"]
        o = ODSKI(q["X"], Grid(q["m"], q["lo"], q["hi"], q.get("interp", "cubic")), q["ell"],
                  q["sf"], q["noise_value"], q["noise_grad"])
        A = _dense_matrix(o, True)
        r = {"n": int(q["X"].shape[0]), "rtol": SUB_RTOL, "probes": SUB_PROBES,
             "depth": SUB_DEPTH}
        if "x" in sub:
            xd = chol_solve(A, q["y"])
            nq = float(np.linalg.norm(q["y"]))
            r["solve"] = {"iters": sub["iters"], "relres_gpu": sub["relres"],
                          "relres_oracle": float(np.linalg.norm(q["y"] - A @ sub["x"]) / nq),
                          "backward_diff_vs_direct": float(np.linalg.norm(A @ (sub["x"] - xd)) / nq)}
        else:
            r["solve"] = {"error": sub.get("solve_error")}
        Lo, _, _ = pivoted_cholesky(o.kgrad_diag(), o.kgrad_row, sub["rank"], pivots=sub["piv"])
        Pc = QRPreconditioner(Lo, o.noise)
        if "logdet" in sub:
            Z = preconditioned_probes(777, Pc, SUB_PROBES)
            est, se_o, _, _ = slq_logdet_z(o.mvm, Pc, Z, depth=SUB_DEPTH, rtol=1e-15,
                                           maxit=SUB_DEPTH)
            exact = chol_logdet(A)
            r["logdet"] = {"gpu": sub["logdet"], "oracle_same_probes": float(est),
                           "rel_err_same_probes": float(abs(sub["logdet"] - est) / abs(est)),
                           "exact_dense": float(exact),
                           "gpu_minus_exact_in_se": float((sub["logdet"] - exact) / sub["logdet_se"])}
        else:
            r["logdet"] = {"error": sub.get("logdet_error")}
        if "grad" in sub:
            Z = preconditioned_probes(31, Pc, SUB_PROBES)
            _, _, go = mll_grad_hutchinson_direct(o, q["y"], Pc, Z, factored=True)
            ge = mll_grad_dense(o, q["y"], factored=True)
            g = np.array(sub["grad"])
            r["grad"] = {"gpu": g.tolist(), "oracle_same_probes": go.tolist(),
                         "max_rel_err_same_probes": float(np.max(np.abs(g - go)) / np.max(np.abs(go))),
                         "exact_dense": ge.tolist()}
        else:
            r["grad"] = {"error": sub.get("grad_error")}
        out["subsample_" + sub["prec"]] = r
    return out


SWEEP = ((100_000, 256), (1_000_000, 256), (10_000_000, 1024), (30_000_000, 1024))


def run_sweep(args):
    """Scatter and gather bandwidth against the HBM model at growing n (the
    terrain shape: points uniform in [0,1]^2, grid over [-0.05, 1.05]^2,
    l = 0.05), FP64 and FP32 (mixed) vectors, s = 1 and 8.  Inputs are made
    on the device (seeded); the values do not change the work."""
    import torch
    from paper_1810_12283_gb300 import DSKI
    dev = torch.device("cuda", 0)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs") or 6800.0
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    pts = []
    reps = 10
    for n, g in SWEEP:
        if n > args.sweep_max_n:
            continue
        gen = torch.Generator(device=dev)
        gen.manual_seed(n)
        X = torch.rand((n, 2), generator=gen, device=dev, dtype=torch.float64)
        M = g * g
        for prec in ("fp64", "mixed_3xtf32"):
            op = DSKI(X, [g, g], [-0.05, -0.05], [1.05, 1.05], [0.05, 0.05], 1.0, 1e-3, 1e-3,
                      prec=prec)
            elem = 8 if prec == "fp64" else 4
            for s in (1, 8):
                v = torch.randn((s, op.N), generator=gen, device=dev, dtype=torch.float64).to(op.dtype)
                out = torch.empty_like(v)
                for _ in range(3):
                    op.mvm(v, out=out)
                torch.cuda.synchronize()
                op.profile_start()
                for i in range(reps):
                    flush.fill_(i & 255)
                    op.mvm(v, out=out)
                st = op.profile_stop()[0]
                t_sc = st["scatter"][0] / reps / 1e3
                t_ga = st["gather"][0] / reps / 1e3
                bs = scatter_bytes(n, 2, M, s, elem)
                bg = gather_bytes(n, 2, M, s, elem)
                pts.append({"n": n, "grid": g, "prec": prec, "s": s,
                            "scatter_us": round(t_sc * 1e6, 2), "gather_us": round(t_ga * 1e6, 2),
                            "scatter_gbs": round(bs / t_sc / 1e9, 1),
                            "gather_gbs": round(bg / t_ga / 1e9, 1),
                            "scatter_frac": round(bs / t_sc / 1e9 / hbm, 3),
                            "gather_frac": round(bg / t_ga / 1e9 / hbm, 3)})
                del v, out
            op.close()
        del X
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "D-SKI scatter / gather bandwidth vs the HBM model (sweep over n)",
                      "unit": "GB/s", "peak_hbm_gbs": hbm,
                      "l2": "flushed before each timed MVM (256 MiB write)", "reps": reps,
                      "points": pts}), flush=True)
    return 0


KUU_SWEEP = (256, 512, 1024)


def run_kuu_sweep(args):
    """The products with K_UU at growing grids (d = 2, g x g nodes over
    [-0.05, 1.05]^2, l = 0.05 * 256 / g so that every grid resolves its kernel
    alike, 200,000 points uniform in [0,1]^2): device time of the d mode
    products per MVM (stage timers, kron stage), dense Kronecker factors on
    the FP64 units, on the tensor cores (FP64_TC, m <= 256) and the
    Toeplitz/FFT form, with the FFT MVM's relative difference from the dense
    FP64 MVM.  Inputs are made on the device (seeded)."""
    import torch
    from paper_1810_12283_gb300 import DSKI
    dev = torch.device("cuda", 0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    reps = 20
    n = 200_000
    pts = []
    gen = torch.Generator(device=dev)
    gen.manual_seed(17)
    X = torch.rand((n, 2), generator=gen, device=dev, dtype=torch.float64)
    v = torch.randn(3 * n, generator=gen, device=dev, dtype=torch.float64)
    for g in KUU_SWEEP:
        ell = 0.05 * 256 / g
        outs = {}
        for prec, kuu in (("fp64", "dense"), ("fp64_tc", "dense"), ("fp64", "fft")):
            if prec == "fp64_tc" and g > 256:
                continue
            op = DSKI(X, [g, g], [-0.05, -0.05], [1.05, 1.05], [ell, ell], 1.0, 1e-3, 1e-3,
                      prec=prec, kuu=kuu)
            out = torch.empty_like(v)
            for _ in range(3):
                op.mvm(v, out=out)
            torch.cuda.synchronize()
            op.profile_start()
            for i in range(reps):
                flush.fill_(i & 255)
                op.mvm(v, out=out)
            st = op.profile_stop()[0]
            outs[(prec, kuu)] = out.clone()
            op.close()
            pts.append({"grid": g, "prec": prec, "kuu": kuu,
                        "kron_us_per_mvm": round(1e3 * st["kron"][0] / reps, 2),
                        "mvm_us": round(1e3 * sum(x[0] for x in st.values()) / reps, 2)})
        ref = outs[("fp64", "dense")]
        d = float(torch.linalg.norm(outs[("fp64", "fft")] - ref) / torch.linalg.norm(ref))
        pts.append({"grid": g, "fft_vs_dense_fp64_rel": d})
    print(json.dumps({"metric": "K_UU mode products per D-SKI MVM: dense Kronecker vs Toeplitz/FFT",
                      "unit": "us", "n": n, "reps": reps,
                      "l2": "flushed before each timed MVM (256 MiB write)", "points": pts}),
          flush=True)
    return 0


PRECOND_ELLS = (0.05, 0.1, 0.2, 0.4)
PRECOND_SIGMAS = (1e-3, 1e-2, 1e-1)   # noise standard deviations (variance sigma^2)
SURFACE_RANKS = (0, 25, 50, 100, 128)


def run_precond_sweep(args):
    """The preconditioning experiment of App. C, and the same diagnosis on the
    3-D surface workload.

    1. D-SKI on Franke's function (2,000 points, 96^2 grid, s_f = 1):
       iterations of plain CG and of PCG with the rank-100 pivoted Cholesky
       preconditioner to relative residual 1e-4, over length scales and noise
       levels; a solve that does not reach it within the cap is reported as
       not converged.
    2. The implicit-surface workload (27,500 points, 64^3 grid, l = 0.2):
       pivoted-Cholesky ranks 0 (plain CG) .. 128 at its noise 1e-4 and at
       larger noises, each solve capped at --surface-maxit iterations: the
       iterations to 1e-4 and the relative residual reached, and the time per
       iteration.  Inputs are seeded and synthetic."""
    import torch
    from paper_1810_12283_gb300 import DSKI
    from synth import workloads as W
    dev = torch.device("cuda", 0)
    prec = args.prec

    def solve(p, rank, rtol, maxit):
        X = torch.tensor(p["X"], device=dev)
        op = DSKI(X, p["m"], p["lo"], p["hi"], p["ell"], p["sf"], p["noise_value"],
                  p["noise_grad"], prec=prec)
        pc = op.pivchol(rank) if rank > 0 else None
        y = torch.tensor(p["y"], device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            _, it, rr = op.solve(y, pc, rtol=rtol, maxit=maxit, allow_not_converged=True)
            err = None
        except Exception as e:   # noqa: BLE001 -- reported
            it, rr, err = [None], [None], str(e)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if pc is not None:
            pc.close()
        op.close()
        out = {"iters": it[0], "relres": rr[0], "s": round(dt, 3),
               "converged": rr[0] is not None and rr[0] <= rtol}
        if err:
            out["error"] = err
        return out

    franke = []
    for ell in PRECOND_ELLS:
        for sig in PRECOND_SIGMAS:
            p = W.franke2d(ell=ell, noise=sig * sig)
            row = {"ell": ell, "sigma": sig}
            for rank, key in ((0, "cg"), (100, "pcg_rank100")):
                row[key] = solve(p, rank, 1e-4, args.franke_maxit)
            franke.append(row)
    surface = []
    base = W.surface3d()
    for noise, ranks in ((1e-4, SURFACE_RANKS), (1e-3, (0, 100)), (1e-2, (0, 100))):
        p = dict(base, noise_value=noise, noise_grad=noise)
        for rank in ranks:
            r4 = solve(p, rank, 1e-4, args.surface_maxit)
            r8 = solve(p, rank, 1e-8, args.surface_maxit)
            surface.append({"noise": noise, "rank": rank, "to_1e-4": r4, "to_1e-8": r8,
                            "s_per_iter": r8["s"] / max(r8["iters"] or 1, 1)})
    print(json.dumps({"metric": "CG vs pivoted-Cholesky PCG iterations (App. C) and the 3-D "
                                "surface rank sweep",
                      "mode": prec, "franke2d": {"n": 2000, "grid": "96x96", "rtol": 1e-4,
                                                  "maxit": args.franke_maxit, "cells": franke},
                      "surface3d": {"n": int(base["X"].shape[0]), "grid": "64^3", "ell": 0.2,
                                    "maxit": args.surface_maxit, "runs": surface}}),
          flush=True)
    return 0


def run_surface(args):
    """The implicit-surface workloads (points on a bumpy sphere, 64^3 grid over
    [-1.4, 1.4]^3, l = 0.2, noise 1e-4, rank-100 pivoted Cholesky):
      * 27,500 points: the PCG solve of y to relative residual 1e-8 and the
        SLQ log determinant with 31 probes at Lanczos depth 30;
      * 55,000 points: the log marginal likelihood of Eq. 1 and its gradient
        with respect to (log l_1..3, log s_f, log s_n) through the autograd
        Function (one batched PCG of the solve and 16 probes to --surface-rtol,
        the SLQ log determinant and the grid adjoint).
    Each step is timed with the host clock around device-synchronised calls
    (inputs resident on the device).  Inputs are seeded and synthetic."""
    import torch
    from paper_1810_12283_gb300 import DSKI, mll_function
    from synth import workloads as W
    dev = torch.device("cuda", 0)
    prec = args.prec
    out = {"mode": prec}

    def build(p):
        X = torch.tensor(p["X"], device=dev)
        return DSKI(X, p["m"], p["lo"], p["hi"], p["ell"], p["sf"], p["noise_value"],
                    p["noise_grad"], prec=prec)

    def clock(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    p = W.surface3d()
    op = build(p)
    pc, t_pc = clock(lambda: op.pivchol(RANK))
    y = torch.tensor(p["y"], device=dev)
    (x, it, rr), t_solve = clock(lambda: op.solve(y, pc, rtol=RTOL, maxit=args.surface_solve_maxit,
                                                  allow_not_converged=True))
    (ld, se), t_slq = clock(lambda: op.logdet(pc, probes=31, depth=30, seed=777))
    out["surface3d_27500"] = {"pivchol_s": t_pc, "solve": {"iters": it[0], "relres": rr[0],
                                                           "s": t_solve, "rtol": RTOL},
                              "slq": {"logdet": ld, "stderr": se, "probes": 31, "depth": 30,
                                      "s": t_slq}}
    pc.close()
    op.close()
    q = W.surface3d_big()
    op = build(q)
    d = op.d
    theta = torch.tensor([math.log(v) for v in q["ell"]] + [math.log(q["sf"]),
                         0.5 * math.log(q["noise_value"])], dtype=torch.float64,
                         requires_grad=True)
    yq = torch.tensor(q["y"], device=dev)

    def grad_step():
        L = mll_function(theta, op, yq, rank=RANK, probes=16, seed=777, rtol=args.surface_rtol,
                         maxit=args.surface_solve_maxit)
        (g,) = torch.autograd.grad(L, theta)
        return float(L.detach()), g.tolist()

    try:
        (L, g), t_grad = clock(grad_step)
        out["surface3d_55000_grad"] = {"mll": L, "grad": g, "s": t_grad, "probes": 16,
                                       "rtol": args.surface_rtol,
                                       "theta": "log l_1..3, log s_f, log s_n"}
    except Exception as e:   # noqa: BLE001 -- reported
        out["surface3d_55000_grad"] = {"error": str(e)}
    op.close()
    print(json.dumps({"metric": "implicit-surface workloads: solve to 1e-8, 31-probe SLQ, "
                                "55,000-point gradient of Eq. 1", **out}), flush=True)
    return 0


MULTI_INSTANCES = 256
MULTI_ORACLE_SAMPLE = 16


def run_multi(args):
    """--multi: print multi_instance_result's line."""
    print(json.dumps(multi_instance_result(args)), flush=True)
    return 0


def multi_instance_result(args):
    """The uneven multi-instance workload: 256 independent GP-with-gradient
    problems (d in {2, 3}, n log-uniform in [200, 5000], 48^2 or 24^3 grids,
    rank-32 pivoted Cholesky, PCG to 1e-6).  Default: the handles and
    preconditioners are built on --multi-workers host threads (one stream
    each), then one persistent launch solves all 256 (a CTA per system);
    --multi-streams: every problem also solves on its own stream.  Reports
    instances/s over the whole batch (set-up included), the set-up and solve
    split, p50/p99 per-instance solve time, the convergence count, and (the
    oracle leg, on the host cores) ||y - K~_oracle x|| / ||y|| on a seeded
    sample of the instances.  Inputs are seeded and synthetic."""
    import torch
    import numpy as np
    from paper_1810_12283_gb300 import launch_count
    from paper_1810_12283_gb300.batch import solve_many
    from synth import workloads as W
    count = args.multi_instances
    probs = [W.multi_instance(i) for i in range(count)]
    persistent = not args.multi_streams
    # warm-up: one instance of each dimension (kernel loading, tuner)
    solve_many([probs[0], probs[1]], rank=32, rtol=1e-6, maxit=40000, prec=args.prec,
               workers=2, persistent=persistent, cluster=args.multi_cluster)
    torch.cuda.synchronize()
    launches0 = launch_count()
    tim = {}
    t0 = time.perf_counter()
    res = solve_many(probs, rank=32, rtol=1e-6, maxit=args.multi_maxit, prec=args.prec,
                     workers=args.multi_workers, persistent=persistent, timings=tim,
                     cluster=args.multi_cluster)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    secs = sorted(r["seconds"] for r in res)
    conv = sum(1 for r in res if r["error"] is None and r["relres"] <= 1e-6)
    its = sorted(r["iters"] for r in res if r["error"] is None)
    line = {"metric": f"multi-instance D-SKI PCG throughput ({count} uneven problems, rtol 1e-6)",
            "unit": "instances/s", "value": count / wall, "wall_s": wall,
            "mode": args.prec, "workers": args.multi_workers,
            "solver": ("one persistent launch, a cluster of CTAs per system "
                       "(dski_pcg_solve_batch)" if persistent
                       else "a stream per system (dski_pcg_solve)"),
            "cluster": (args.multi_cluster or 4) if persistent else None,
            "p50_s": secs[len(secs) // 2], "p99_s": secs[min(len(secs) - 1, int(0.99 * len(secs)))],
            "max_s": secs[-1],
            "per_instance_time": ("solve time inside the persistent launch (device clock)"
                                  if persistent else "wall time of the instance on its stream"),
            "converged": conv, "instances": count, "maxit": args.multi_maxit,
            "iters_p50": its[len(its) // 2] if its else None,
            "iters_max": its[-1] if its else None,
            "gpu_launches": launch_count() - launches0,
            "errors": sorted({r["error"] for r in res if r["error"]})[:3]}
    if tim:
        line["setup_s"] = tim["setup_s"]
        line["solve_s"] = tim["solve_s"]
        line["solve_only_instances_per_s"] = count / tim["solve_s"]
        # the persistent kernel is bound by the FP64 units: its algorithmic
        # FP64 flops (batch_iter_flops x iterations, summed over the systems)
        # over the launch's wall time, against this GPU's measured DGEMM rate
        flops = 0.0
        for q, r in zip(probs, res):
            n, d = q["X"].shape
            flops += r["iters"] * batch_iter_flops(n, d, int(np.prod(q["m"])), int(sum(q["m"])), 32)
        fp64 = measure_peaks("cuda")["fp64_tflops"]
        ach = flops / tim["solve_s"] / 1e12
        C = line["cluster"]
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        line["roofline"] = {"bound": "alu", "achieved": ach, "peak": fp64, "unit": "TFLOP/s",
                            "frac": ach / fp64, "traffic": None,
                            "kernel": "k_batch_pcg (FP64 SIMT; one launch)",
                            "peak_source": "measured in this run: cuBLAS DGEMM 8192^3, best of 3",
                            "flops": flops}
        # share of the launch's SM-time spent inside solves (a cluster of C
        # CTAs holds C SMs while it solves a system)
        line["sm_busy_fraction"] = sum(r["seconds"] for r in res) * C / (tim["solve_s"] * sms)
    if not args.no_cpu_baseline:
        from oracle.dski import DSKI as ODSKI, Grid
        rng = np.random.default_rng(11)
        sample = sorted(rng.choice(count, min(count, MULTI_ORACLE_SAMPLE), replace=False).tolist())
        errs = []
        for i in sample:
            q, r = probs[i], res[i]
            if r["x"] is None:
                errs.append(None)
                continue
            o = ODSKI(q["X"], Grid(q["m"], q["lo"], q["hi"]), q["ell"], q["sf"],
                      q["noise_value"], q["noise_grad"])
            errs.append(float(np.linalg.norm(q["y"] - o.mvm(r["x"].numpy())) /
                              np.linalg.norm(q["y"])))
        line["oracle_check"] = {"sample": sample, "relres_oracle": errs,
                                "max": max(e for e in errs if e is not None)}
    return line


def run_reference(args, p):
    rank, ws, dist = dist_init()
    if rank != 0:
        return 0
    # the oracle PCG is extrapolated to the iteration count FP64 PCG needs
    # for this system (measured on GB300; --ref-iters): a full oracle solve
    # would take ~35 minutes of CPU time
    iters = args.ref_iters
    src = ("FP64 PCG iterations of this system to 1e-8 measured on GB300"
           if iters == FP64_TERRAIN_ITERS else "--ref-iters")
    steps = []
    for _ in range(max(args.steps, 1)):
        steps.append(cpu_baseline(p, iters, src,
                                  budget_s=max(4.0, 60.0 / (args.steps + args.warmup))))
    v = statistics.median(s["value"] for s in steps)
    cb = dict(steps[0])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(p["X"].shape[0], p["interp"], p["kuu"]), "l2": "n/a (CPU)"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp64_tc", choices=["fp64_tc", "fp64", "mixed_3xtf32"])
    ap.add_argument("--compare", default="fp64,mixed_3xtf32",
                    help="comma-separated modes timed beside the headline mode, one step each "
                         "(the headline's warm-up steps have run every kernel they use); "
                         "fp64 / fp64_tc run to the tolerance, the mixed modes are capped at "
                         "min(1.5x the headline iterations, 30000)")
    ap.add_argument("--maxit", type=int, default=400000)
    ap.add_argument("--n", type=int, default=100_000)
    ap.add_argument("--ref-iters", type=int, default=FP64_TERRAIN_ITERS,
                    help="reference arm: PCG iterations to extrapolate the oracle's "
                         "per-iteration time to")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--interp", default="cubic", choices=["cubic", "quintic"],
                    help="interpolation stencil (Keys cubic, 4^d; the paper's quintic, 6^d)")
    ap.add_argument("--sweep", action="store_true",
                    help="instead of the solve step: scatter / gather bandwidth at n = 1e5 .. 3e7")
    ap.add_argument("--sweep-max-n", type=int, default=30_000_000)
    ap.add_argument("--kuu-sweep", action="store_true",
                    help="instead of the solve step: K_UU products, dense vs FFT, grids 256..1024")
    ap.add_argument("--precond-sweep", action="store_true",
                    help="instead of the solve step: App. C's CG vs PCG iteration counts "
                         "(Franke, 2000 points) and a preconditioner-rank sweep on the 3-D "
                         "surface workload")
    ap.add_argument("--franke-maxit", type=int, default=50000)
    ap.add_argument("--surface", action="store_true",
                    help="instead of the solve step: the implicit-surface solve, SLQ and the "
                         "55,000-point gradient")
    ap.add_argument("--surface-rtol", type=float, default=1e-8)
    ap.add_argument("--surface-solve-maxit", type=int, default=600000)
    ap.add_argument("--multi", action="store_true",
                    help="instead of the solve step: the 256-instance uneven workload")
    ap.add_argument("--multi-workers", type=int, default=8)
    ap.add_argument("--multi-instances", type=int, default=MULTI_INSTANCES,
                    help="--multi: the first K instances of the workload (default 256)")
    ap.add_argument("--multi-maxit", type=int, default=40000,
                    help="--multi: iteration cap per system (a small cap bounds a profiling run)")
    ap.add_argument("--multi-cluster", type=int, default=0, choices=[0, 1, 2, 4, 8],
                    help="--multi: CTAs per system in the persistent launch (0: default)")
    ap.add_argument("--no-multi", action="store_true",
                    help="default step: leave out the nested 256-instance measurement")
    ap.add_argument("--multi-streams", action="store_true",
                    help="--multi: solve each instance on its own stream instead of in one "
                         "persistent launch")
    ap.add_argument("--surface-maxit", type=int, default=20000)
    ap.add_argument("--kuu", default="dense", choices=["dense", "fft"],
                    help="products with K_UU: dense Kronecker factors or Toeplitz/FFT")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    args.steps = max(args.steps, 1)

    from synth import workloads as W
    p = W.terrain2d(n=args.n)
    p["interp"] = args.interp
    p["kuu"] = args.kuu
    SN = stencil_nodes(args.interp)
    if args.sweep:
        return run_sweep(args)
    if args.kuu_sweep:
        return run_kuu_sweep(args)
    if args.precond_sweep:
        return run_precond_sweep(args)
    if args.multi:
        return run_multi(args)
    if args.surface:
        return run_surface(args)
    if args.impl == "reference":
        return run_reference(args, p)

    import torch
    rank, ws, dist = dist_init()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1810_12283_gb300 import DSKI, launch_count

    n, d = p["X"].shape
    N = n * (d + 1)
    M = int(np.prod(p["m"]))
    X = torch.tensor(p["X"], device=dev)
    y = torch.tensor(p["y"], device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(prec, X_, y_, prof=False, maxit=None):
        op = DSKI(X_, p["m"], p["lo"], p["hi"], p["ell"], p["sf"], p["noise_value"],
                  p["noise_grad"], prec=prec, interp=args.interp, kuu=args.kuu)
        if prof:
            op.profile_start()
        pc = op.pivchol(RANK)
        try:
            x, it, rr = op.solve(y_, pc, rtol=RTOL, maxit=maxit or args.maxit,
                                 allow_not_converged=True)
        except Exception as e:   # breakdown of a mode that cannot resolve the system
            if prof:
                op.profile_stop()
            pc.close()
            op.close()
            raise e
        st = op.profile_stop()[0] if prof else None
        return op, pc, x, it[0], rr[0], st

    def timed_steps(prec, warm, steps, prof, maxit=None):
        for _ in range(warm):
            op, pc, *_ = step(prec, X, y, maxit=maxit)
            pc.close()
            op.close()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        ms, its, rrs, stages, launches, xlast = [], [], [], None, 0, None
        for i in range(steps):
            flush.fill_(i & 255)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0 = launch_count()
            a.record(stream)
            op, pc, x, it, rr, st = step(prec, X, y, prof=prof, maxit=maxit)
            b.record(stream)
            b.synchronize()
            launches += launch_count() - l0
            ms.append(a.elapsed_time(b))
            its.append(it)
            rrs.append(rr)
            if st is not None:
                stages = st
            xlast = x
            pc.close()
            op.close()
        if dist is not None:
            dist.barrier()
        return ms, its, rrs, stages, launches, xlast

    def mvm_rate(prec, reps=50):
        op = DSKI(X, p["m"], p["lo"], p["hi"], p["ell"], p["sf"], p["noise_value"],
                  p["noise_grad"], prec=prec, interp=args.interp, kuu=args.kuu)
        v = torch.randn(N, device=dev, dtype=op.dtype)
        out = torch.empty_like(v)
        for _ in range(5):
            op.mvm(v, out=out)
        torch.cuda.synchronize()

        def timed(profiled):
            # the stage timers' events would add to the MVM's own time, so the
            # MVM is timed with them off and the stage split taken in a second,
            # profiled pass
            if profiled:
                op.profile_start()
            tot = 0.0
            for i in range(reps):
                flush.fill_(i & 255)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                op.mvm(v, out=out)
                b.record(stream)
                b.synchronize()
                tot += a.elapsed_time(b)
            return tot, (op.profile_stop()[0] if profiled else None)

        tot, _ = timed(False)
        _, st = timed(True)
        op.close()
        per = tot / reps
        elem = 8 if prec in ("fp64", "fp64_tc") else 4
        algo = mvm_bytes(n, d, 1, elem)
        extra = 2 * n * weight_table_bytes(d, elem, SN)
        return {"ms_per_mvm": per, "gbs": algo / (per / 1e3) / 1e9, "algo_bytes": algo,
                "extra_traffic": extra,
                "extra_traffic_note": "per-point stencil weight tables read by scatter and "
                                      "gather, beyond the algorithmic model (not counted in gbs)",
                "stages_us": {k: round(1e3 * v[0] / max(v[2], 1) * v[1] / reps, 2)
                              for k, v in st.items() if v[1]}}

    # timed steps with the stage timers off: the PCG chunks then replay as
    # CUDA graphs (the timers' events would disable them)
    with ClockSampler(local) as clk:
        ms, its, rrs, _, launches, x_head = timed_steps(args.prec, args.warmup, args.steps, False)
    clocks = clk.summary()
    xs = {args.prec: x_head.cpu().numpy()}
    # stage data from one more, untimed step with the timers on, its PCG
    # capped at PROF_ITERS iterations
    prof_iters = min(PROF_ITERS, max(its[-1], 1))
    _, _, _, stages, _, _ = timed_steps(args.prec, 0, 1, True, maxit=prof_iters)
    compare = {}
    for mode in [m for m in args.compare.split(",") if m and m != args.prec]:
        try:
            cap = args.maxit if mode in ("fp64", "fp64_tc") else min(int(1.5 * its[-1]) + 100, 30000)
            msc, itc, rrc, _, _, xc = timed_steps(mode, 0, 1, False, maxit=cap)
            compare[mode] = {"s_per_step": msc[-1] / 1e3, "iters": itc[-1], "relres": rrc[-1],
                             "reached_rtol": rrc[-1] <= RTOL, "iter_cap": cap,
                             "s_per_iter": msc[-1] / 1e3 / max(itc[-1], 1)}
            xs[mode] = xc.cpu().numpy()
        except Exception as e:   # noqa: BLE001 -- reported, not fatal
            compare[mode] = {"error": str(e)}
    mvm = {prec: mvm_rate(prec) for prec in ("fp64", "fp64_tc", "mixed_3xtf32")
           if not (args.kuu == "fft" and prec.startswith("mixed"))}   # FFT: FP64 vectors only

    # end to end through the public calls with host buffers
    Xh = torch.tensor(p["X"]).pin_memory()
    yh = torch.tensor(p["y"]).pin_memory()
    xh = torch.empty(N, dtype=torch.float64).pin_memory()
    flush.fill_(7)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    Xd = Xh.to(dev, non_blocking=True)
    yd = yh.to(dev, non_blocking=True)
    op, pc, x, it_e, rr_e, _ = step(args.prec, Xd, yd)
    xh.copy_(x, non_blocking=True)
    b.record(stream)
    b.synchronize()
    e2e_s = a.elapsed_time(b) / 1e3
    pc.close()
    op.close()

    t_step = reduce_max(dist, statistics.median(ms), dev) / 1e3
    e2e_s = reduce_max(dist, e2e_s, dev)

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs") or 6800.0
    hbm_src = "measured" if peaks.get("hbm_gbs") else "fallback"
    bf16 = peaks.get("bf16_tflops_sustained") or 1700.0
    bf16_src = ("measured" if peaks.get("bf16_tflops_sustained") else "fallback") + \
        " sustained dense BF16 (cuBLAS; the kernel runs inside a long step)"
    gemm = measure_peaks(dev)   # FP64 and TF32 dense-GEMM rates of this GPU, in this run
    fp64_pk = gemm["fp64_tflops"]
    fp64_src = "measured in this run: cuBLAS DGEMM 8192^3, best of 3"
    it_last = its[-1]
    # per stage (profiled step: set-up + prof_iters PCG iterations): mean
    # device time per launch, and per PCG iteration for the iteration stages
    st = {k: v for k, v in stages.items() if v[1]}
    per_launch_ms = {k: v[0] / max(v[2], 1) for k, v in st.items()}
    stage_total_ms = {k: per_launch_ms[k] * v[1] for k, v in st.items()}
    iter_stages = ("scatter", "kron", "gather", "precond", "pcg_vec")
    # Roofline of the kernel the ncu launch list of this command ranks first.
    # FP64: the Kronecker mode product k_mode_simt (one launch per mode
    # product, 2 M m_k FP64 flops) against the measured DGEMM rate.  FP64_TC:
    # the digit-product kernel k_oz_mode, one launch per mode product (the
    # kron stage), the method's 2 M m_k flops against the BF16 tensor pipe it
    # runs on; the rate of the 36 digit-pair BF16 products it issues for them,
    # and the FP64-equivalent rate against the measured DGEMM rate, beside it.
    # Mixed modes: the FP32 scatter against the HBM model.  The FP64 scatter
    # is reported beside (FP64 flops against the measured DGEMM rate).
    roof_scatter = None
    extra = {}
    elem = 8 if args.prec in ("fp64", "fp64_tc") else 4
    if args.prec in ("fp64", "fp64_tc") and args.prec in mvm:
        # one scatter: its stage time in the timed MVM (one scatter per MVM)
        per_sc = mvm[args.prec]["stages_us"]["scatter"] / 1e6
        fl = scatter_flops(n, d, SN)
        bsc = scatter_bytes(n, d, M, 1, 8)
        df = args.prec == "fp64_tc" and d == 2 and SN == 4
        roof_scatter = {"kernel": ("k_scatter_split_df + k_scatter_cells_df + k_scatter_nodes_df "
                                   "(scatter; stencil products in double-float on the FP32 units)"
                                   if df else "k_scatter_prep + k_scatter_ab (scatter)"),
                        "bound": "alu",
                        "achieved": fl / per_sc / 1e12, "peak": fp64_pk, "unit": "TFLOP/s",
                        "frac": fl / per_sc / 1e12 / fp64_pk, "peak_source": fp64_src,
                        "algo_per_launch": fl,
                        "note": ("the method's FP64 flops per scatter over its time, against the "
                                 "measured DGEMM rate" +
                                 ("; the double-float products run on the FP32 units, so the "
                                  "fraction can pass 1" if df else "")),
                        "hbm_view": {"algo_bytes": bsc, "achieved_gbs": bsc / per_sc / 1e9,
                                     "frac_of_hbm": bsc / per_sc / 1e9 / hbm}}
    if args.prec == "fp64":
        per_s = per_launch_ms["kron"] / 1e3
        algo = 2 * M * p["m"][0]
        achieved = algo / per_s / 1e12
        kern, bound, unit, peak, peak_src = ("k_mode_simt (kron, one mode product)", "alu",
                                             "TFLOP/s", fp64_pk, fp64_src)
    elif args.prec == "fp64_tc":
        per_s = per_launch_ms["kron"] / 1e3
        algo = 2 * M * p["m"][0]
        achieved = algo / per_s / 1e12
        kern, bound, unit, peak, peak_src = ("k_oz_mode (kron, one mode product)", "tensor",
                                             "TFLOP/s", bf16, bf16_src)
        extra = {"digit_products": {"algo_per_launch": OZ_PAIRS * algo,
                                    "achieved": OZ_PAIRS * achieved,
                                    "frac": OZ_PAIRS * achieved / bf16,
                                    "note": "the 36 BF16 digit-pair products issued per FP64 "
                                            "product (the tensor pipe's own work)"},
                 "fp64_equivalent": {"achieved": achieved, "peak": fp64_pk,
                                     "frac": achieved / fp64_pk, "peak_source": fp64_src}}
    else:
        per_s = 2 * per_launch_ms["scatter"] / 1e3
        algo = scatter_bytes(n, d, M, 1, 4)
        achieved = algo / per_s / 1e9
        kern, bound, unit, peak, peak_src = ("k_scatter_cells + k_scatter_nodes (scatter)", "hbm",
                                             "GB/s", hbm, hbm_src + " HBM copy bandwidth")
    roofline = {"kernel": kern, "bound": bound, "achieved": achieved, "peak": peak,
                "peak_source": peak_src, "unit": unit, "frac": achieved / peak,
                "traffic": None,
                "traffic_note": "DRAM bytes per launch come from the ncu capture of this kernel "
                                "on the same workload, not from this run",
                "algo_per_launch": algo, "launch_us": per_s * 1e6}
    roofline.update(extra)
    line = {
        "metric": METRIC, "value": t_step, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(n, p["interp"], p["kuu"]), "mode": args.prec,
                   "l2": "flushed before each timed step (256 MiB write)",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "solve": {"iters": its, "relres": rrs, "s_per_iter": t_step / it_last,
                  "reached_rtol": all(r <= RTOL for r in rrs)},
        "compare": compare,
        "profiled_step": {"pcg_iters": prof_iters,
                          "note": "stage timers on (CUDA graphs off); not part of value",
                          "stage_us_per_launch": {k: round(1e3 * v, 2) for k, v in per_launch_ms.items()},
                          "stage_launches": {k: v[1] for k, v in st.items()},
                          "stage_us_per_iter": {k: round(1e3 * stage_total_ms[k] / prof_iters, 1)
                                                for k in iter_stages if k in stage_total_ms}},
        "mvm": mvm,
        "peaks": {"hbm_gbs": hbm, "hbm_source": hbm_src, "bf16_tflops_sustained": bf16,
                  "fp64_tflops": fp64_pk, "tf32_tflops": gemm["tf32_tflops"],
                  "gemm_source": fp64_src.replace("DGEMM", "GEMM (DGEMM; TF32 FP32 GEMM)")},
        "roofline_scatter": roof_scatter,
        "roofline": roofline,
        "e2e": {"value": e2e_s, "unit": UNIT, "h2d_bytes_per_step": (n * d + N) * 8,
                "d2h_bytes_per_step": N * 8, "iters": it_e, "relres": rr_e},
        "gpu_launches": launches // args.steps,
        "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle leg: the GPU's results on a seeded subsample first (GPU
        # work, untimed), then the oracle on the host cores
        subs = []
        for mode in dict.fromkeys([args.prec, "fp64"]):
            subs.append(gpu_subsample_run(DSKI, p, mode, dev))
        built = oracle_operator(p)
        if "fp64" in compare and "iters" in compare["fp64"]:
            ref_it, ref_src = compare["fp64"]["iters"], "this run's FP64 PCG iteration count"
        else:
            ref_it, ref_src = it_last, f"this run's {args.prec} PCG iteration count"
        line["cpu_baseline"] = cpu_baseline(p, ref_it, ref_src, built=built)
        line["oracle_check"] = oracle_check(p, built, xs, subs)
    if rank == 0 and not args.no_multi and args.interp == "cubic" and args.kuu == "dense":
        # the many-instance workload (256 uneven systems in one persistent
        # launch), after the timed region: its own line's fields, nested
        try:
            line["multi_instance"] = multi_instance_result(args)
        except Exception as e:   # noqa: BLE001 -- reported, never fatal to the line
            line["multi_instance"] = {"error": str(e)[:300]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
