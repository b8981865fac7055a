"""The N > 1 path of bench.py on CPU: world_size-2 gloo process group, the
timed region taken as the maximum over ranks and the job throughput as the
units of all replicas over that time (independent lysosomes or seeds per
rank, no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds = 1.0 + rank  # rank 1 is the slower one
    t = bench.max_over_ranks_of(seconds, world, "cpu")
    out[rank] = (t, bench.job_throughput(6.4e7, t, world), bench.dist_env()[:2])
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, value, (r, w) = res[rank]
        assert t == 2.0                     # slowest rank's time
        assert value == 2 * 6.4e7 / 2.0      # all units over that time
        assert (r, w) == (rank, world)
