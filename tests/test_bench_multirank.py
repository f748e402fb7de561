"""Host logic of the N-rank benchmark path with world_size 2 on CPU (gloo):
each rank steps its own envs (no data-path collective); the timing is the
slowest rank's and the rate counts every rank's env-steps."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_info() == (rank, world, rank)
    ms = 100.0 + 50.0 * rank                       # rank 1 is the slow one
    slow = bench.max_over_ranks(ms, world, "cpu")
    out[rank] = (slow, bench.whole_job_rate(256, 8, world, slow))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_all_env_steps():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for r in range(world):
        slow, rate = res[r]
        assert slow == 150.0
        assert rate == pytest.approx(256 * 8 * 2 / 0.150)
