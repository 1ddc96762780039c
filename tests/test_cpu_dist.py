"""The multi-rank path of the benchmark on CPU (gloo, world size 2): each rank
advances its own shard (ids offset by rank, no collective in the data path);
only the timing (max over ranks) and the work (sum) are reduced."""
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


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    from paper_1608_06356_gb300 import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    st, _, _ = W.chi_target(1000 + 500 * rank, seed=rank)
    ids = st["id"] + bench.rank_id_offset(rank)
    ms = 10.0 + 5.0 * rank
    ps = float(len(ids))
    t, total = bench.reduce_over_ranks(dist, ms, ps, "cpu")
    gathered = [None] * world
    dist.all_gather_object(gathered, (int(ids.min()), int(ids.max())))
    out[rank] = (t, total, gathered)
    dist.destroy_process_group()


def test_two_rank_reduction_and_disjoint_ids():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        t, total, ranges = res[r]
        assert t == 15.0
        assert total == 1000 + 1500
        (a0, a1), (b0, b1) = ranges
        assert a1 < b0  # shards never share an id
