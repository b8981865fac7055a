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


def _failing_worker(rank, world, port, out):
    import datetime
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    import bench
    if rank == 1:
        out[rank] = "raised"
        raise RuntimeError("rank 1 fails before the timing reduction")
    try:
        bench.max_over_ranks_of(1.0, world, "cpu")
        out[rank] = "no error"
    except Exception as e:  # the lost peer surfaces as an error, not a hang
        out[rank] = "error: " + type(e).__name__


def test_a_failed_rank_ends_the_others_collective():
    # failure injected on the host: one rank raises, the survivor's next
    # collective ends with an error within the process-group timeout
    world = 2
    ctx = mp.get_context("spawn")
    with mp.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_failing_worker, args=(r, world, port, out))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        alive = [p.is_alive() for p in procs]
        for p in procs:
            if p.is_alive():
                p.kill()
        res = dict(out)
    assert not any(alive)
    assert procs[1].exitcode != 0
    assert res.get(1) == "raised"
    assert res.get(0, "").startswith("error")
