"""The multi-GPU bench's cross-rank logic on two CPU processes (gloo): every
rank runs its own batch, and only a barrier and the maximum of the timed
seconds cross ranks."""
import json
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    ranks = bench.Ranks("gloo", "cpu")
    ranks.barrier()
    seconds = 1.0 + rank          # the slower rank decides the timed region
    slowest = ranks.max(seconds)
    rate = ranks.aggregate_rate(units_per_rank=300.0, seconds=seconds)
    ranks.barrier()
    ranks.close()
    q.put((rank, slowest, rate))


def test_two_gloo_ranks_take_the_slowest_rank_and_aggregate_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slowest, rate in out:
        assert slowest == 2.0                 # max over ranks
        assert rate == pytest.approx(2 * 300.0 / 2.0)   # all ranks' units / slowest time
