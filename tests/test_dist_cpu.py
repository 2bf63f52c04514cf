"""The multi-GPU path of bench.py, run on the CPU: world_size-2 gloo ranks.

The graph build shards by event with no exchange step (replicas); the only
collectives are the timing reductions.  Each rank must build different events
(no two ranks share a seed), the step time taken is the max over ranks and the
event count is the sum."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    args = bench.parse_args(["--gpus", str(world)])
    r, w, local, pg = bench.dist_setup(args)
    assert (r, w) == (rank, world) and pg is not None
    seeds = [bench.synth.seed_of("c3", r * 4 + e) for e in range(4)]
    t = bench.max_over_ranks(pg, 1.0 + rank)
    n = bench.sum_over_ranks(pg, 10.0 * (rank + 1))
    bench.barrier(pg)
    out[rank] = (seeds, t, n)
    pg.destroy_process_group()


@pytest.mark.timeout(180)
def test_two_gloo_ranks_replicas_and_timing_reduction():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank_main, args=(i, world, port, out)) for i in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=150)
        codes = [p.exitcode for p in procs]
        res = dict(out)
    assert codes == [0, 0], codes
    s0, t0, n0 = res[0]
    s1, t1, n1 = res[1]
    assert not set(s0) & set(s1)           # ranks build different events
    assert t0 == t1 == 2.0                 # max over ranks
    assert n0 == n1 == 30.0                # events summed over ranks


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    import bench
    called = []
    monkeypatch.setattr(bench, "run_cpu_baseline", lambda *a, **k: called.append(1))
    assert bench.reference_arm(bench.parse_args(["--impl", "reference"]), rank=1, world=2) == 0
    assert not called
