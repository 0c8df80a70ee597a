"""Host-side logic of the multi-rank benchmark (replicas of independent
solves), exercised with world_size 2 on CPU over gloo."""
import os
import socket

import pytest

torch = pytest.importorskip('torch')


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    os.environ['MASTER_ADDR'] = '127.0.0.1'
    os.environ['MASTER_PORT'] = str(port)
    dist.init_process_group('gloo', rank=rank, world_size=world)
    import bench
    # rank r took (r + 1) seconds for (10 r + 5) units
    secs, units = bench.aggregate(float(rank + 1), float(10 * rank + 5), world)
    out.put((rank, secs, units))
    dist.destroy_process_group()


def test_aggregate_max_time_and_summed_units():
    import torch.multiprocessing as mp
    ctx = mp.get_context('spawn')
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, secs, units in res:
        assert secs == 2.0          # the slowest replica sets the time
        assert units == 20.0        # 5 + 15 units over both ranks


def test_aggregate_single_rank_is_identity():
    import bench
    assert bench.aggregate(1.5, 7.0, 1) == (1.5, 7.0)
