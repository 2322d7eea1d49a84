"""Host-side logic of bench.py (no GPU): the max-over-ranks reduction of the
N > 1 path on two gloo ranks, and the algorithmic byte counts the roofline
fields are computed from."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), DSKI_BENCH_BACKEND="gloo")
    import bench
    r, ws, d = bench.dist_init()
    assert (r, ws) == (rank, world)
    got = bench.reduce_max(d, 1.5 + 2.0 * rank, torch.device("cpu"))
    out.put((rank, got))
    d.barrier()
    d.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(2))
    assert res == {0: 3.5, 1: 3.5}


def test_single_process_reduce_is_identity():
    import bench
    assert bench.reduce_max(None, 2.25, torch.device("cpu")) == 2.25


def test_algorithmic_byte_counts():
    """The MVM's algorithmic HBM bytes: v read by the scatter and by the noise
    term, out written (3 N s elements), the geometry (cell id + d fractions,
    g = 4 + b d bytes) read by scatter and gather; the grid stays in L2."""
    import bench
    n, d = 100_000, 2
    N = n * (d + 1)
    assert bench.geometry_bytes(2, 4) == 12 and bench.geometry_bytes(3, 4) == 16
    assert bench.mvm_bytes(n, d, 1, 4) == 3 * N * 4 + 2 * n * 12
    assert bench.mvm_bytes(n, d, 1, 8) == 3 * N * 8 + 2 * n * (4 + 8 * d)
    # the terrain value of the byte model: ~6 MB per FP32 MVM
    assert abs(bench.mvm_bytes(n, d, 1, 4) - 6.0e6) < 1e3
    # weight tables (S weights + S derivative weights per dimension) are extra traffic
    assert bench.weight_table_bytes(d, 4) == 4 * 2 * 4 * d


def test_scatter_byte_count():
    import bench
    n, d, M = 100_000, 2, 65_536
    assert bench.scatter_bytes(n, d, M, 1, 8) == 3 * n * 8 + n * (4 + 2 * 8) + M * 8


def test_gather_byte_count():
    import bench
    n, d, M = 100_000, 2, 65_536
    assert bench.gather_bytes(n, d, M, 1, 4) == M * 4 + 2 * 3 * n * 4 + n * (4 + 2 * 4)


def test_scatter_flop_count():
    import bench
    assert bench.scatter_flops(100_000, 2) == 100_000 * 83


def test_quintic_stencil_counts_and_workload_names():
    # the quintic stencil (6 nodes per dimension): 2 * 6 * d weights per
    # point, 36 node-point pairs per point in the d = 2 node pass
    import bench
    n, d, M = 1000, 2, 256 * 256
    assert bench.stencil_nodes("cubic") == 4 and bench.stencil_nodes("quintic") == 6
    assert bench.weight_table_bytes(d, 8, 6) - bench.weight_table_bytes(d, 8) == (2 * 6 - 2 * 4) * d * 8
    assert bench.scatter_flops(n, d, 6) == n * (3 + 6 * 3 + 6 + 36 * 4)
    name = bench.workload_name(100_000)
    assert "interp" not in name and "kuu" not in name
    assert bench.workload_name(100_000, "quintic", "fft").endswith("interp=quintic kuu=fft")


def test_batch_iteration_flop_count():
    import bench
    # d = 2, cubic: scatter 4 (3 + 1) + 16 (3 + 1) = 80 and gather
    # 4 * 16 + 6 * 4 = 88 flops per point; 48^2 grid: 2 M (48 + 48)
    assert bench.batch_iter_flops(10, 2, 48 * 48, 96, 32) == 10 * 168 + 2 * 2304 * 96 + 30 * 145
    # d = 3: scatter 20 + 64 + 256 = 340, gather 256 + 96 + 32 = 384
    assert bench.batch_iter_flops(5, 3, 24 ** 3, 72, 0) == 5 * 724 + 2 * 13824 * 72 + 20 * 17


def test_multi_instance_workload_recipe():
    # the 256-system workload: d in {2, 3}, n log-uniform in [200, 5000], points
    # in the unit box, 48^2 or 24^3 grids over [-0.1, 1.1]^d, rank 32, rtol 1e-6,
    # values then the d gradient blocks as the target; seeded (same i, same system)
    import numpy as np
    from synth import workloads as W
    seen = set()
    for i in range(64):
        p = W.multi_instance(i)
        n, d = p["X"].shape
        seen.add(d)
        assert d in (2, 3) and 200 <= n <= 5000
        assert tuple(p["m"]) == ((48, 48) if d == 2 else (24, 24, 24))
        assert tuple(p["lo"]) == (-0.1,) * d and tuple(p["hi"]) == (1.1,) * d
        assert p["X"].min() >= 0.0 and p["X"].max() <= 1.0
        assert p["y"].shape == (n * (d + 1),) and np.all(np.isfinite(p["y"]))
        assert p["rank"] == 32 and p["rtol"] == 1e-6
        assert 0.05 <= float(np.atleast_1d(p["ell"])[0]) <= 0.3
    assert seen == {2, 3}
    q = W.multi_instance(5)
    assert np.array_equal(q["X"], W.multi_instance(5)["X"])
