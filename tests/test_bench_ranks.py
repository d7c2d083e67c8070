"""Host logic of the multi-rank bench path, on CPU with two gloo ranks.

With N GPUs every rank steps its own replica of the workload.  No data-path collective is
involved, because the on-line stage of independent source batches does not shard.  The one
exchange is the max over ranks of the timed seconds, which turns per-rank times into the
whole-job throughput.  Here it runs with the gloo backend on 127.0.0.1.
"""
import multiprocessing as mp
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, seconds, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        rate, slowest = bench.whole_job_rate(100.0, seconds[rank], world, dist, "cpu")
        q.put((rank, rate, slowest))
    finally:
        dist.destroy_process_group()


def test_single_rank_rate_is_units_over_time():
    assert bench.whole_job_rate(300.0, 1.5, 1) == (200.0, 1.5)


@pytest.mark.parametrize("seconds", [(1.0, 2.0), (4.0, 0.5)])
def test_two_gloo_ranks_take_the_slowest_rank(seconds):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, seconds, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    out = sorted(q.get(timeout=5) for _ in range(2))
    slow = max(seconds)
    for rank, rate, slowest in out:
        assert slowest == slow
        assert rate == pytest.approx(2 * 100.0 / slow)
