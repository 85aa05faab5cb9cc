"""The N > 1 path of the benchmark on CPU: two gloo ranks run the same
host-side logic the GPU ranks run (independent task per rank, max-over-ranks
job time, whole-job value), with no data-path collective."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_local = 1.0 + rank             # rank 1 is the slower one
        t_job = bench.job_seconds(t_local, world)
        value = bench.job_value(world, 10, 1e9, t_job)
        out[rank] = (bench.rank_task(rank), t_job, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_job_time():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] != res[1][0]                     # independent problems
    assert res[0][1] == res[1][1] == 2.0              # slowest rank's time
    assert res[0][2] == res[1][2] == 2 * 10 * 1e9 / 2.0
