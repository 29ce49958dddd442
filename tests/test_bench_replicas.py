"""The multi-process (replicas) bookkeeping of bench.py on CPU with the gloo backend: every rank
gets the slowest rank's time, and the whole-job value counts the units of all ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, ws: int, port: int, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        ms = bench.replica_time(100.0 * (rank + 1), ws, "cpu")  # rank r took 100 (r + 1) ms
        q.put((rank, ms, bench.replica_value(1000.0, 10, ws, ms)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_max_time_and_sum_the_work():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(ws))
    for rank, ms, value in got:
        assert ms == 200.0                       # the slower rank's time
        assert value == 2 * 10 * 1000.0 / 0.2    # both ranks' units over that time


def test_single_process_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_time(12.5, 1) == 12.5
    assert bench.replica_value(100.0, 4, 1, 12.5) == 4 * 100.0 / 0.0125
