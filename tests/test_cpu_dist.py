"""The multi-rank path of the benchmark on CPU (gloo, world size 2): each rank
advances its own shard (ids offset by rank, no collective in the data path);
only the timing (max over ranks), the work (sum) and, at the end of the run,
the event counters and the 64-bin photon spectrum (sums, status bits OR-ed)
are reduced.  The QED step on each rank is the oracle's (CPU); the reduced
counters and spectrum must equal those of one step over the union of the
shards, exactly (particles are independent and their random numbers are keyed
by id)."""
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


def _step_worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import numpy as np
    import bench
    import oracle as O
    from paper_1608_06356_gb300 import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    st, _, _ = W.chi_target(600, seed=77)
    lo, hi = (0, 250) if rank == 0 else (250, 600)  # uneven shards of one ensemble
    sub = {k: v[lo:hi] for k, v in st.items()}
    cfg = O.make_config(dt=0.05, seed=9)
    e = O.Species(4 * (hi - lo), -1.0, per_particle_fields=True).load(**sub)
    g = O.Species(16 * (hi - lo), 0.0, per_particle_fields=True, with_alive=True)
    lc, _ = O.step(cfg, O.per_particle_fields(), e, O.Species(1, 1.0, True), g, 3)
    c = {"emit_events": lc.events, "pair_events": 0, "substeps": lc.substeps, "dropped": lc.dropped,
         "domain": 0, "deferred": 0, "status": 1 if rank == 1 else 0, "hist": list(lc.hist)}
    out[rank] = bench.reduce_counters(dist, c, "cpu")
    dist.destroy_process_group()


def test_two_rank_counter_and_spectrum_reduction_equals_the_union():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle as O
    from paper_1608_06356_gb300 import workloads as W
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_step_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=600)
            assert p.exitcode == 0
        res = dict(out)
    st, _, _ = W.chi_target(600, seed=77)
    cfg = O.make_config(dt=0.05, seed=9)
    e = O.Species(2400, -1.0, per_particle_fields=True).load(**st)
    g = O.Species(9600, 0.0, per_particle_fields=True, with_alive=True)
    lc, _ = O.step(cfg, O.per_particle_fields(), e, O.Species(1, 1.0, True), g, 3)
    for r in range(world):
        red = res[r]
        assert red["emit_events"] == lc.events > 50
        assert red["substeps"] == lc.substeps
        assert red["hist"] == list(lc.hist)
        assert red["status"] == 1  # OR over ranks
