"""Benchmark of the D-SKI hot path on one GB300 (or N independent replicas).

Workload: the terrain stand-in -- n = 100,000 points uniform in [0,1]^2 with
values and gradients of a 512-feature random Fourier field (N = 300,000
rows), SE length scale 0.05, noise 1e-3, 256 x 256 grid over [-0.05, 1.05]^2.
Inputs are synthetic and seeded (``synth.workloads.terrain2d``).

A step is one D-SKI MVM K~ v (Sec. 3.1) of one fresh right-hand side in the
mixed (3xTF32 / FP32) mode, with the FP64 mode timed beside it.  The L2 is
flushed (a 256 MiB write) between timed steps, outside the timed events.

Printed: one JSON line (rank 0).  ``--impl reference`` times the plain FP64
CPU oracle on the host cores instead (the reference arm of this project).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "D-SKI MVM effective HBM GB/s (mixed 3xTF32/FP32), terrain n=100k d=2 grid 256^2"
UNIT = "GB/s"
WORKLOAD = "terrain2d n=100000 d=2 N=300000 grid=256x256 s=1"


def mvm_bytes(n, d, M, s, elem):
    """Algorithmic HBM bytes of one MVM: v read by scatter and by the noise
    term, out written, the per-point geometry (cell id + d fractions) read by
    scatter and gather, the grid written by scatter and read by gather."""
    N = n * (d + 1)
    geo = n * (4 + elem * d)
    return s * (3 * N * elem + 2 * M * elem) + 2 * geo


def scatter_bytes(n, d, M, s, elem):
    N = n * (d + 1)
    return s * (N * elem + M * elem) + n * (4 + elem * d)


def gather_bytes(n, d, M, s, elem):
    N = n * (d + 1)
    return s * (M * elem + 2 * N * elem) + n * (4 + elem * d)


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
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
        for ln in getattr(self, "lines", []):
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
    backend = os.environ.get("DSKI_BENCH_BACKEND", "nccl")
    dist.init_process_group(backend)
    return dist.get_rank(), dist.get_world_size(), dist


def reduce_max(dist, value, device):
    """Max over ranks of a host float (a no-op on one process)."""
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


def cpu_baseline(p, budget_s=12.0):
    """The FP64 oracle MVM on the host cores, on a bounded number of MVMs."""
    from oracle.dski import DSKI as ODSKI, Grid
    t0 = time.perf_counter()
    op = ODSKI(p["X"], Grid(p["m"], p["lo"], p["hi"]), p["ell"], p["sf"], p["noise_value"],
               p["noise_grad"])
    t_setup = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    reps, t_mvm = 0, 0.0
    while t_mvm < budget_s and reps < 200:
        v = rng.normal(size=op.N)
        t0 = time.perf_counter()
        op.mvm(v)
        t_mvm += time.perf_counter() - t0
        reps += 1
    per = t_mvm / reps
    M = int(np.prod(p["m"]))
    n, d = p["X"].shape
    gbs = mvm_bytes(n, d, M, 1, 8) / per / 1e9
    return {"value": gbs, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
            "sample": f"{reps} FP64 oracle MVMs of the full terrain operator "
                      f"({per * 1e3:.1f} ms each; setup {t_setup:.1f} s untimed)",
            "ms_per_mvm": per * 1e3}


def run_reference(args, p):
    rank, ws, dist = dist_init()
    if rank != 0:
        return 0
    cb = cpu_baseline(p, budget_s=max(2.0, 60.0 / max(args.steps + args.warmup, 1)))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": cb["ms_per_mvm"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "flushed between steps"},
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=100_000)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    from synth import workloads as W
    p = W.terrain2d(n=args.n)
    if args.impl == "reference":
        return run_reference(args, p)

    import torch
    rank, ws, dist = dist_init()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1810_12283_gb300 import DSKI, launch_count

    n, d = p["X"].shape
    M = int(np.prod(p["m"]))
    X = torch.tensor(p["X"], device=dev)
    ops = {prec: DSKI(X, p["m"], p["lo"], p["hi"], p["ell"], p["sf"], p["noise_value"],
                      p["noise_grad"], prec=prec)
           for prec in ("mixed_3xtf32", "fp64")}
    N = ops["fp64"].N
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    rng = torch.Generator(device=dev)
    rng.manual_seed(1234 + rank)
    stream = torch.cuda.current_stream(dev)

    def timed(op, steps, prof):
        vs = [torch.randn(N, device=dev, dtype=op.dtype, generator=rng) for _ in range(4)]
        out = torch.empty(N, device=dev, dtype=op.dtype)
        for i in range(args.warmup):
            op.mvm(vs[i % 4], out=out)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        l0 = launch_count()
        if prof:
            op.profile_start()
        for i in range(steps):
            flush.fill_(i & 255)
            ev[i][0].record(stream)
            op.mvm(vs[i % 4], out=out)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        stages = op.profile_stop()[0] if prof else None
        launches = launch_count() - l0
        ms = sum(a.elapsed_time(b) for a, b in ev)
        if dist is not None:
            dist.barrier()
        return ms, launches, stages

    res = {}
    with ClockSampler(local) as clk:
        for prec, op in ops.items():
            res[prec] = timed(op, args.steps, prof=True)
    clocks = clk.summary()

    # end to end through the public call with pinned host buffers
    op = ops["mixed_3xtf32"]
    hv = torch.randn(N, dtype=torch.float32).pin_memory()
    ho = torch.empty(N, dtype=torch.float32).pin_memory()
    dv = torch.empty(N, device=dev, dtype=torch.float32)
    for _ in range(args.warmup):
        dv.copy_(hv, non_blocking=True)
        ho.copy_(op.mvm(dv), non_blocking=True)
    torch.cuda.synchronize()
    e_ms = 0.0
    for i in range(args.steps):
        flush.fill_(i & 255)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dv.copy_(hv, non_blocking=True)
        ho.copy_(op.mvm(dv), non_blocking=True)
        b.record(stream)
        b.synchronize()
        e_ms += a.elapsed_time(b)

    ms_mixed = reduce_max(dist, res["mixed_3xtf32"][0], dev)
    ms_fp64 = reduce_max(dist, res["fp64"][0], dev)
    e_ms = reduce_max(dist, e_ms, dev)
    by_mixed = mvm_bytes(n, d, M, 1, 4)
    by_fp64 = mvm_bytes(n, d, M, 1, 8)
    value = ws * by_mixed * args.steps / (ms_mixed / 1e3) / 1e9
    e2e = ws * by_mixed * args.steps / (e_ms / 1e3) / 1e9

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs")
    peak_note = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    st = res["mixed_3xtf32"][2]
    # dominant kernel of the mixed MVM
    dom = max(("scatter", "gather", "kron"), key=lambda k: st[k][0])
    per_launch_ms = st[dom][0] / max(st[dom][1], 1)
    if dom == "scatter":
        algo = scatter_bytes(n, d, M, 1, 4)
    elif dom == "gather":
        algo = gather_bytes(n, d, M, 1, 4)
    else:
        algo = 2 * M * 4 * d   # each mode product reads and writes the grid
    achieved = algo / (per_launch_ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "flushed between steps (256 MiB write)",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "fp64": {"ms_per_mvm": ms_fp64 / args.steps,
                 "gbs": ws * by_fp64 * args.steps / (ms_fp64 / 1e3) / 1e9,
                 "stages_ms": {k: v[0] / args.steps for k, v in res["fp64"][2].items()}},
        "stages_ms_mixed": {k: v[0] / args.steps for k, v in st.items()},
        "roofline": {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm,
                     "peak_source": peak_note, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": None, "algo_bytes_per_launch": algo},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": N * 4,
                "d2h_bytes_per_step": N * 4},
        "gpu_launches": res["mixed_3xtf32"][1],
        "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p)
        line["cpu_baseline"].pop("ms_per_mvm", None)
    if rank == 0:
        print(json.dumps(line), flush=True)
    for op in ops.values():
        op.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
