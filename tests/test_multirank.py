"""CPU test of bench.py's multi-rank (replica) aggregation with two gloo ranks:
the timed region is the maximum over ranks and the value counts the work of
every rank."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t, v = bench.aggregate(100.0 + 50.0 * rank, ws, pairs_step=1e12, steps=3, device="cpu")
    q.put((rank, t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_takes_max_and_counts_all_work():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == pytest.approx(150.0)
        assert v == pytest.approx(2 * 1e12 * 3 / 0.150)
