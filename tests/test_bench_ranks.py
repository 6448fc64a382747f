"""Multi-rank (replica) aggregation of bench.py on CPU with the gloo backend, world size 2."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 1.5 + r seconds and finished 3 + r requests (7 r of them certified)
        t, counts = bench.combine_ranks(dist, 1.5 + rank, [3 + rank, 7 * rank], "cpu")
        out.put((rank, t, counts))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, counts in got:
        assert t == pytest.approx(2.5)          # the slowest rank's time
        assert counts == [7, 7]                 # summed over ranks
