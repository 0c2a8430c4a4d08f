"""The multi-rank bench path on CPU: two gloo ranks, each with its own time;
the job's throughput counts every rank's rays over the slowest rank's time
(replicas; no data-path collective besides this timing reduction)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 * (rank + 1)  # rank 1 is the slowest
    value, total_ms = bench.job_throughput(local_ms, rays_per_rank=1_000_000, world=world, dist=dist)
    q.put((rank, value, total_ms, bench.rank_info()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_throughput_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(world))
    for rank, value, total_ms, info in res:
        assert total_ms == 200.0  # max over ranks
        assert value == pytest.approx(2 * 1_000_000 / 0.2 / 1e6)  # whole job: 10 Mrays/s
        assert info == (rank, 0, world)


def test_launch_count_includes_the_sort():
    # gpu_launches counts the sort's kernels when the options sort: histogram,
    # scan of 8192-bin tiles (plus a second pass past one tile), scatter, and the
    # gather of the hits
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    d = (9, 9, 9)
    assert bench.trace_launches(None, d) == 1
    assert bench.trace_launches({"sort_cell_log2": 0}, d) == 1
    assert bench.trace_launches({"sort_cell_log2": 6}, d) == 5   # 8 x 8^3 = 4096 bins: one tile
    assert bench.trace_launches({"sort_cell_log2": 4}, d) == 6   # 8 x 32^3 bins: several tiles
    assert bench.trace_launches({"sort_cell_log2": 9}, d) == 5   # one cell: 8 bins
