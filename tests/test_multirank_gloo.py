"""The N > 1 bench path on CPU: two gloo ranks reduce their work and times the way bench.py does for
GPU replicas (units summed over ranks, time = the slowest rank's)."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, results):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r did 100 (r + 1) units in (r + 1) seconds
        value, seconds, units = bench.job_throughput(100 * (rank + 1), float(rank + 1))
        results[rank] = (value, seconds, units)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_throughput_reduction():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        results = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, results)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        got = dict(results)
    for r in range(world):
        value, seconds, units = got[r]
        assert units == 300.0
        assert seconds == 2.0
        assert value == 150.0
