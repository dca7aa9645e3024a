"""The N-GPU bench path on CPU: ranks are independent replicas (seed +
rank), and the whole-job figure is every rank's tuples over the slowest
rank's time.  Two gloo ranks on 127.0.0.1; nothing here touches a GPU."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        secs, derived = bench.over_ranks(1.0 + rank, 10 * (rank + 1), dist, "cpu")
        spec = bench.WORKLOADS["tc-er-1000-1500"]
        edges = bench.make_program(spec, seed_offset=rank).edb["edge"]
        out.put((rank, secs, derived, edges.tobytes()))
    finally:
        dist.destroy_process_group()


def test_two_replicas_reduce_to_the_whole_job():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(2):
        rank, secs, derived, edges = q.get(timeout=120)
        got[rank] = (secs, derived, edges)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        assert got[r][0] == pytest.approx(2.0)  # the slowest rank
        assert got[r][1] == 30                  # every rank's tuples
    assert got[0][2] != got[1][2]               # replicas draw their own instance


def test_one_rank_is_unchanged():
    import bench
    assert bench.over_ranks(3.5, 7, None, "cpu") == (3.5, 7)
