"""Multi-rank aggregation of bench.py on CPU (gloo, world size 2): every rank
solves its own problem, so the job's time is the slowest rank's and its work is
the sum over ranks; no collective touches the data path."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank
    res = bench.aggregate_ranks(dist, ms, 2 * ms, cycles=6 + rank, e2e_cycles=12 + rank)
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        ms, ms_e2e, cyc, e2e = out[r]
        assert ms == 15.0 and ms_e2e == 30.0
        assert cyc == 13.0 and e2e == 25.0
