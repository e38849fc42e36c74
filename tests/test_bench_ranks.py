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


def test_roofline_uses_the_roofline_bytes_per_cell_update():
    """Host arithmetic of the bench's roofline: algorithmic bytes per cell-update are 92 (FP32 MUSCL
    and WAF), 68 (FP32 first-order HLLC), 172 and 124 in FP64; the line's frac is the whole step at
    those bytes over the measured copy rate, and the dominant kernel is reported by the same count."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert [bench.roofline_bytes(s, "fp32") for s in ("muscl", "waf", "hllc")] == [92, 92, 68]
    assert [bench.roofline_bytes(s, "fp64") for s in ("muscl", "hllc")] == [172, 124]
    prof = {"prep": (0.2 * 10, 10), "flux": (0.3 * 10, 10)}        # (total ms, launches)
    r = bench.roofline_entry("muscl", 1_000_000, 0.5, prof, "split", 5000.0, "measured", None)
    assert abs(r["achieved"] - 92 * 1e6 / 0.5e-3 / 1e9) < 1e-9 and abs(r["frac"] - r["achieved"] / 5000.0) < 1e-12
    assert r["kernel"]["name"] == "k_flux" and abs(r["kernel"]["ms"] - 0.3) < 1e-12
    assert abs(r["kernel"]["achieved"] - 92 * 1e6 / 0.3e-3 / 1e9) < 1e-9
    assert r["own_bytes"]["flux"]["bytes_per_cell"] == 116 and r["own_bytes"]["prep"]["bytes_per_cell"] == 100


def test_own_bytes_follow_the_wet_fraction_and_the_source_hash_ignores_comments(tmp_path, monkeypatch):
    """A dry cell stores and reads no face values: the split MUSCL kernels' own bytes are the mix
    at the state's wet fraction (prep 100 B wet / 8 B dry, flux 116 / 68 in FP32); and the hash
    that keys stored ncu counters changes with the kernel code, not with its comments."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.algo_bytes("prep", "muscl", "fp32", 0.5) == 54 and bench.algo_bytes("flux", "muscl", "fp32", 0.5) == 92
    assert bench.algo_bytes("prep", "muscl", "fp32") == 100 and bench.algo_bytes("flux", "muscl", "fp32", 0.0) == 68
    prof = {"prep": (2.0, 10), "flux": (3.0, 10)}
    r = bench.roofline_entry("muscl", 1_000_000, 0.5, prof, "split", 5000.0, "measured", 123.0, wet=0.5)
    assert r["own_bytes"]["prep"]["bytes_per_cell"] == 54 and r["own_bytes"]["wet_fraction"] == 0.5
    assert r["traffic"] == 123.0 and "traffic_source" in r
    src = tmp_path / "k.cu"
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", ("k.cu",))
    src.write_text("int f() { return 1; }  // one\n")
    a = bench.kernel_source_sha()
    src.write_text("/* prose */\nint f()  {\n  return 1;   // another comment\n}\n")
    assert bench.kernel_source_sha() == a
    src.write_text("int f() { return 2; }\n")
    assert bench.kernel_source_sha() != a
