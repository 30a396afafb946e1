"""The benchmark's multi-rank host logic on CPU ranks (gloo, world size 2): the
timing is the maximum over ranks and the whole-job value counts every rank's
bytes over that time.  Replicas exchange nothing else."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        times = [3.0, 7.5]
        got = bench.max_over_ranks(times[rank])
        value = bench.whole_job_value(1e9, 10, world, got)
        out.put((rank, got, value))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_value_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, got, value in res:
        assert got == 7.5
        # 2 ranks x 10 steps x 1 GB over 7.5 ms
        assert value == pytest.approx(2 * 10 * 1e9 / 7.5e-3 / 1e9)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(4.25) == 4.25
    assert bench.whole_job_value(2e9, 4, 1, 1.0) == pytest.approx(8000.0)
