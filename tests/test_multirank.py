"""The replicas path of bench.py on two CPU ranks (gloo): rank discovery from
the launcher's environment, the max-over-ranks time and the whole-job value."""
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


def _rank(rank, world, port, times, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        t = bench.max_over_ranks(times[rank], dist, "cpu")
        dist.barrier()
        pick = bench.agree_on_rank0({"config": f"chosen by rank {rank}"}, dist)
        out[rank] = (ws, r, local, t, bench.whole_job_value(45, 100, ws, t), pick)
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_whole_job_value():
    world, port = 2, _free_port()
    times = [12.5, 20.0]                      # ms: rank 1 is the slow one
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, times, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ws, r, local, t, value, pick = res[rank]
        assert pick == {"config": "chosen by rank 0"}   # every replica runs rank 0's selection
        assert (ws, r, local) == (world, rank, rank)
        assert t == 20.0                      # every rank reports the slowest rank's time
        assert value == pytest.approx(2 * 45 * 100 * world / 0.020)


def test_single_process_defaults(monkeypatch):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
