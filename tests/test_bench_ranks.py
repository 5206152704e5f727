"""The replica aggregation of bench.py under torch.distributed with two gloo
ranks on the CPU: the reported time is the slowest rank's, the work is the
sum over ranks, and value = total field evaluations / slowest time."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, loc = bench.dist_env()
    ms = [1200.0, 1500.0][rank]               # rank 1 is the slower replica
    evals, accepted = [600, 580][rank], [100, 97][rank]
    res = bench.reduce_over_ranks(dist, ms, evals, accepted, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, (w, r, loc), res))


def test_two_gloo_ranks_take_the_slowest_time_and_the_total_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, env, (ms_max, evals_all, acc_all) in results:
        assert env == (2, rank, rank)
        assert ms_max == 1500.0
        assert evals_all == 1180.0 and acc_all == 197.0
    value = results[0][2][1] / (results[0][2][0] / 1e3)
    assert value == pytest.approx(1180.0 / 1.5)


def test_single_process_passes_through():
    import bench
    assert bench.reduce_over_ranks(None, 10.0, 5, 2, "cpu") == (10.0, 5.0, 2.0)
