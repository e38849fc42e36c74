"""The benchmark's multi-rank path on CPU: two gloo ranks (one process per rank, as torchrun runs
them) reduce the slowest rank's time and the job's cells; each rank draws its own river."""
import multiprocessing as mp
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world)
        ws, r, local = bench.dist_env()
        ms_local = 10.0 + 5.0 * rank                 # rank 1 is the slower one
        cells = 1000 + rank                          # replicas may differ in size
        value, ms = bench.job_throughput(cells, 7, ms_local, dist, "cpu")
        w, grid = bench.river_workload(rank, 0.0005)  # a few thousand cells
        q.put((rank, ws, r, value, ms, float(w.z.sum()), w.n_cells))
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:                           # report instead of hanging the parent
        q.put((rank, "error", repr(e)))


def test_two_gloo_ranks_reduce_time_and_cells():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        item = q.get(timeout=240)
        assert item[1] != "error", item
        out[item[0]] = item
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        _, ws, rr, value, ms, zsum, n = out[r]
        assert ws == 2 and rr == r
        assert ms == 15.0                            # the slowest rank's time on every rank
        assert value == pytest.approx((1000 + 1001) * 7 / 15e-3)
    assert out[0][5] != out[1][5]                    # each rank its own river (own seed)
    assert out[0][6] == out[1][6]                    # of the same size


def test_single_process_needs_no_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.job_throughput(500, 4, 2.0)
    assert ms == 2.0 and value == pytest.approx(500 * 4 / 2e-3)


def test_step_byte_counts_follow_the_wet_fraction():
    """Host arithmetic of the bench's whole-step figures: the split step moves the flux kernel's
    116 B plus prep's 56 B (dry) to 100 B (wet) per cell; the fused kernel 68 B."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.algo_bytes("flux", "muscl", "fp32") == 116 and bench.algo_bytes("prep", "muscl", "fp32") == 100
    assert bench.algo_bytes("fused", "muscl", "fp32") == 68 and bench.algo_bytes("flux", "hllc", "fp32") == 68
    for wet, per_cell in ((0.0, 172.0), (0.5, 194.0), (1.0, 216.0)):
        r = bench.ensemble_roofline("split", 1_000_000, 1.0, wet)
        assert r["algo_bytes_per_cell"] == per_cell
        assert abs(r["achieved"] - per_cell * 1e6 / 1e-3 / 1e9) < 1e-9 and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert bench.ensemble_roofline("fused", 10, 1.0, 0.3)["algo_bytes_per_cell"] == 68.0
