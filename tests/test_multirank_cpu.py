"""Host-side multi-rank logic of the benchmark on CPU (gloo, world size 2):
each rank runs its own lattice (weak scaling, no data-path collective); the
job time is the slowest rank's and the value counts every rank's updates."""
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


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_max, value = bench.job_value(10.0 + 5.0 * rank, 1e9)
    out.put((rank, t_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_job_value_takes_slowest_rank_and_all_updates():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, value in res:
        assert t_max == pytest.approx(15.0)
        assert value == pytest.approx(2 * 1e9 / 15e-3)


def test_job_value_single_process():
    import bench
    assert bench.job_value(20.0, 4e9) == (20.0, pytest.approx(2e11))
