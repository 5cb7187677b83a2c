"""Host logic of the multi-GPU bench on CPU: two gloo ranks, each timing a
different amount, must both see the slowest rank's time, and the reported
throughput is the units of all ranks over that time (weak scaling, one frame per
rank, no collective on the data path)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench._env_rank()
        my_ms = 100.0 + 50.0 * rank
        slow = bench.max_over_ranks(my_ms, w, "cpu")
        dist.barrier()
        q.put((r, w, lr, slow, bench.job_throughput(1000.0, w, slow)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_the_slowest_time_and_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[0] for g in got] == [0, 1] and all(g[1] == 2 for g in got)
    for g in got:
        assert g[3] == pytest.approx(150.0)
        assert g[4] == pytest.approx(2 * 1000.0 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_throughput(540000 * 100, 1, 1000.0) == pytest.approx(5.4e7)
