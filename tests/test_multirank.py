"""Replica (weak-scaling) logic of bench.py on CPU: two gloo ranks get disjoint shards of the
seeded instance stream whose union is the single-rank stream, and the job time is the
slowest rank's time.  No GPU and no collective on the solver's data path."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out, root):
    import sys
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r = bench.shard_range(5, rank)
    specs = bench.workload(5, rank)
    params = [(p.N[0], p.h_terms[0].coef, p.measured) for p in specs]
    ms = bench.max_over_ranks(10.0 * (rank + 1), world)
    out[rank] = (list(r), params, ms)
    dist.destroy_process_group()


def test_two_rank_shards_and_max_time():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import bench
    from workloads import configs
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out, root)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    r0, p0, ms0 = out[0]
    r1, p1, ms1 = out[1]
    assert set(r0).isdisjoint(r1) and sorted(r0 + r1) == list(range(10))
    single = configs.kerr_batch(B=10, T=bench.HORIZON, dt=bench.DT)
    ref = [(p.N[0], p.h_terms[0].coef, p.measured) for p in single]
    assert p0 + p1 == ref
    assert ms0 == ms1 == 20.0
