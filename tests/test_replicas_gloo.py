"""The multi-GPU path of bench.py is N independent replicas: no collective on
the data path, only the timing reduction.  Checked here with two gloo ranks
on the CPU: every rank gets the slowest rank's time, and the whole-job rate
counts the builds of all ranks within it."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks([0.25, 0.75][rank], dist, "cpu")
    dist.barrier()
    q.put((rank, t, bench.whole_job_rate(world, 10, t)))
    dist.destroy_process_group()


def test_replica_timing_reduction_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [0.75, 0.75]
    assert all(abs(o[2] - 2 * 10 / 0.75) < 1e-12 for o in out)


def test_whole_job_rate_single_rank():
    import bench
    assert bench.whole_job_rate(1, 20, 2.0) == pytest.approx(10.0)
