"""Multi-process host logic of bench.py on CPU: two gloo ranks stand in for
two GPUs.  Every rank solves its own replica, so the whole-job rate is the
units all ranks processed over the slowest rank's time; the barriers around
the timed region must complete on every rank."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, units, seconds, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    r, local, w = bench.dist_env()
    assert (r, local, w) == (rank, rank, world)
    ranks = bench.Ranks(world, torch.device("cpu"), backend="gloo")
    try:
        ranks.barrier()
        rate, slowest = ranks.rate(units[rank], seconds[rank])
        ranks.barrier()
        out.put((rank, rate, slowest))
    finally:
        dist.destroy_process_group()


def _run(world, units, seconds):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, units, seconds, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0] * world, codes
    res = sorted(out.get(timeout=10) for _ in range(world))
    return res


def test_whole_job_rate_two_ranks():
    units, seconds = [3.0, 5.0], [0.5, 2.0]
    res = _run(2, units, seconds)
    for rank, rate, slowest in res:
        assert slowest == 2.0
        assert rate == (3.0 + 5.0) / 2.0


def test_whole_job_rate_equal_replicas_is_weak_scaling():
    # identical replicas: N ranks give N times one rank's rate
    res = _run(2, [64.0, 64.0], [0.25, 0.25])
    for _, rate, slowest in res:
        assert slowest == 0.25 and rate == 2 * 64.0 / 0.25


def test_single_process_is_local():
    sys.path.insert(0, ROOT)
    import bench
    ranks = bench.Ranks(1)
    ranks.barrier()
    assert ranks.rate(10, 2.0) == (5.0, 2.0)
