"""Multi-rank host logic of the replicas-only path on CPU ranks (gloo,
world size 2): every rank runs its own replica of the workload with its own
seed, nothing but the timing and the attempt counts is exchanged, the timed
region is the max over ranks and the attempts add up.  The per-rank work here
is the oracle on a tiny instance (the GPU path is exercised by the -m gpu
tests and by bench.py under torchrun)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    import workloads as W
    inst = W.torus(6, 6, signed=True, seed=0)
    p = dict(R=8, sweeps=2, steps=5, seed=bench.rank_seed(100, rank))
    run = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **p)
    run.step(p["steps"])
    cut, spins = run.best()
    run.close()
    fake_ms = 10.0 * (rank + 1)                     # rank 1 is the slower one
    attempts = p["R"] * inst.n * p["sweeps"] * p["steps"]
    ms, total = bench.reduce_over_ranks(dist, fake_ms, attempts, device="cpu")
    g = [None] * world
    dist.all_gather_object(g, (int(cut), spins.tolist()))
    dist.destroy_process_group()
    out.put((rank, ms, total, g, attempts))


def test_two_replica_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    res.sort()
    import bench
    import oracle
    import workloads as W
    inst = W.torus(6, 6, signed=True, seed=0)
    for rank, ms, total, gathered, attempts in res:
        assert ms == 20.0                            # max over ranks
        assert total == world * attempts             # sum over ranks
        # each rank's result is the oracle run with that rank's seed alone
        for r in range(world):
            p = dict(R=8, sweeps=2, steps=5, seed=bench.rank_seed(100, r))
            run = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **p)
            run.step(p["steps"])
            cut, spins = run.best()
            run.close()
            assert gathered[r][0] == cut
            np.testing.assert_array_equal(np.array(gathered[r][1]), spins)
    # the ranks ran different replicas (different seeds)
    assert bench.rank_seed(100, 0) != bench.rank_seed(100, 1)
