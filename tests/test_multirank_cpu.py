"""The multi-GPU reporting path of bench.py ("replicas only": every rank runs
its own transforms, the job rate counts all ranks' pixels over the slowest
rank's time), exercised with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [100.0, 250.0][rank]
    rate, total = bench.whole_job_rate(local_ms, 1_000_000, 10, world,
                                       bench.reduce_max_fn(dist, world, "cpu"))
    q.put((rank, rate, total))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, total in res:
        assert total == 250.0
        assert rate == pytest.approx(1_000_000 * 10 * 2 / 0.25 / 1e9)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    rate, total = bench.whole_job_rate(50.0, 2_000_000, 4, 1, bench.reduce_max_fn(None, 1, "cpu"))
    assert total == 50.0 and rate == pytest.approx(2_000_000 * 4 / 0.05 / 1e9)
