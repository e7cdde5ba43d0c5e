"""One population split over CPU ranks (gloo, world size 2 and 4).

Every rank holds a block of the population's slots; ``run_step`` (the
package's exchange: all-gather of the energies, the plan from the parent
map, all-to-all of the migrating replicas, all-gather after the sweeps) moves
the data, and the oracle does each rank's own part: the population step on
the gathered energies, the cluster moves and sweeps of its own slots, M* and
the controller.  Rows outside a rank's block are overwritten with a constant
row before every iteration, so only the replicas the exchange delivers can
reach an own slot.  The split run must equal the single-process oracle run
bit for bit: spins, energies, parents, counts, the controller and its M*
history, M* and its configuration; the NCM counters add up over the ranks.
The runs cover resampling across block edges, cluster moves, reheats and a
restart that re-draws the population."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

CASES = {
    "ising_ncm": dict(R=32, sweeps=2, steps=150, beta0=0.5, beta1=6.0, stagnation=1, z_rst=120, cooldown_tau=5,
                      seed=3),
    "potts": dict(kind=1, R=16, sweeps=2, steps=90, beta0=0.5, beta1=5.0, stagnation=1, z_rst=70,
                  cooldown_tau=4, seed=4),
    "sa": dict(R=16, sweeps=2, steps=30, beta0=0.5, beta1=3.0, resample=0, seed=5),
}


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _instance():
    import workloads as W
    return W.torus(14, 14, signed=True, seed=2)


class OracleShard:
    """A rank's part of the split population, computed by the oracle (CPU):
    the oracle holds all R rows, but only its own block and the rows the
    exchange delivered are valid."""

    def __init__(self, inst, rank, nranks, params):
        import oracle
        import paper_2606_25203_gb300 as pg
        self.oracle = oracle
        self.params = oracle.make_params(**params)
        self.run = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **params)
        self.R, self.n = self.params["R"], inst.n
        self.rank, self.nranks = rank, nranks
        self.base, self.count = pg.pamc_shard_range(self.R, nranks, rank)
        self.lo, self.hi = self.base, self.base + self.count
        self.run.set_own(self.lo, self.hi)
        self.redraws = self.params["z_rst"] > 0 and self.params["restart_reinit"] != 0
        self.E_own = torch.zeros(self.count, dtype=torch.int64)
        self.E_all = torch.zeros(self.R, dtype=torch.int64)
        self.e_all_valid = False
        self.moved = 0
        self.poison = np.full((self.R, self.n), 1 if self.params["kind"] == 0 else 0, dtype=np.int8)

    def _own_energy(self, out):
        out.copy_(torch.from_numpy(self.run.energy()[self.lo:self.hi].copy()))

    def rows(self, k):
        return torch.zeros(int(k) * self.n, dtype=torch.int8)

    def energies(self, E_own):
        self._own_energy(E_own)

    def resample(self, E_all):
        # every other rank's rows become a constant row: an own slot can only
        # get a foreign parent through the exchange
        self.run.set_rows(0, self.poison[:self.lo])
        self.run.set_rows(self.hi, self.poison[self.hi:])
        E = E_all.numpy().copy()
        self.run.set_energies(E)
        c = self.run.ctl()
        if c["z"] > 1 and self.params["resample"]:
            escale = 0.5 if self.params["kind"] == 1 else 1.0
            parent, _ = self.oracle.resample(E, c["delta"], escale, self.params["seed"], c["t"])
        else:
            parent = np.arange(self.R, dtype=np.int32)
        self.parent = parent
        return parent

    def pack(self, rows, send):
        if len(rows):
            send.copy_(torch.from_numpy(self.run.spins()[self.lo + np.asarray(rows)].reshape(-1)))

    def sweep(self, E_all, local_parent, recv, nimports, E_own):
        own_par = self.parent[self.lo:self.hi]
        foreign = np.unique(own_par[(own_par < self.lo) | (own_par >= self.hi)])
        assert len(foreign) == nimports
        got = recv.numpy().reshape(nimports, self.n)
        for g, row in zip(foreign.tolist(), got):
            self.run.set_rows(g, row)
        # the plan's source rows: own rows first, then the received ones
        expect = np.where((own_par >= self.lo) & (own_par < self.hi), own_par - self.lo,
                          self.count + np.searchsorted(foreign, own_par))
        np.testing.assert_array_equal(np.asarray(local_parent), expect)
        self.run.set_energies(E_all.numpy().copy())
        self.run.iter_population()
        self.run.iter_sweeps()
        self._own_energy(E_own)

    def control(self, E_all, E_own):
        self.run.set_energies(E_all.numpy().copy())
        self.run.iter_control()
        self._own_energy(E_own)

    def best(self):
        cut, spins = self.run.best()
        owned = self.run.best_owned()
        return cut, (spins if owned else None), owned


def _rank_main(rank, world, port, case, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2606_25203_gb300 import shard as S
        params = CASES[case]
        shard = OracleShard(_instance(), rank, world, params)
        comm = S.TorchComm()
        for _ in range(params["steps"]):
            S.run_step(shard, comm)
        cut, best = S.best(shard, comm)
        r = shard.run
        par, cnt = r.parents()
        res = dict(rank=rank, lo=shard.lo, hi=shard.hi, spins=r.spins()[shard.lo:shard.hi],
                   E=r.energy()[shard.lo:shard.hi], parent=par, count=cnt, ctl=r.ctl(), hist=r.history(),
                   cut=cut, best=best, moved=shard.moved, targets=r.ncm_targets())
        dist.barrier()
    finally:
        dist.destroy_process_group()
    out.put(res)


def _groups_main(rank, world, port, out):
    """Two populations of R = 16 over two ranks each (subgroups of a world of
    four), with their own seeds, as the benchmark runs several populations
    when one would exceed the population step's size."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2606_25203_gb300 import shard as S
        groups = [dist.new_group([0, 1]), dist.new_group([2, 3])]
        pop, prank = rank // 2, rank % 2
        params = dict(CASES["ising_ncm"], R=16, steps=40, z_rst=30, seed=10 + pop)
        shard = OracleShard(_instance(), prank, 2, params)
        comm = S.TorchComm(groups[pop])
        assert (comm.rank, comm.size) == (prank, 2)
        for _ in range(params["steps"]):
            S.run_step(shard, comm)
        cut, best = S.best(shard, comm)
        res = dict(rank=rank, pop=pop, spins=shard.run.spins()[shard.lo:shard.hi], cut=cut, best=best)
        dist.barrier()
    finally:
        dist.destroy_process_group()
    out.put(res)


def test_two_populations_on_subgroups():
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_groups_main, args=(r, 4, port, q)) for r in range(4)]
    for pr in procs:
        pr.start()
    res = sorted([q.get(timeout=300) for _ in range(4)], key=lambda d: d["rank"])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    inst = _instance()
    for pop in (0, 1):
        params = dict(CASES["ising_ncm"], R=16, steps=40, z_rst=30, seed=10 + pop)
        ref = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **params)
        ref.step(params["steps"])
        part = [r for r in res if r["pop"] == pop]
        np.testing.assert_array_equal(np.concatenate([r["spins"] for r in part]), ref.spins())
        mstar, best = ref.best()
        for r in part:
            assert r["cut"] == mstar
            np.testing.assert_array_equal(r["best"], best)
        ref.close()


def _run_split(case, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, case, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    return sorted(res, key=lambda d: d["rank"])


@pytest.mark.parametrize("case,world", [("ising_ncm", 2), ("ising_ncm", 4), ("potts", 2), ("sa", 4)])
def test_split_population_equals_single_run(case, world):
    import oracle
    params = CASES[case]
    inst = _instance()
    ref = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **params)
    ref.step(params["steps"])
    parts = _run_split(case, world)

    spins = np.concatenate([p["spins"] for p in parts])
    E = np.concatenate([p["E"] for p in parts])
    np.testing.assert_array_equal(spins, ref.spins())
    np.testing.assert_array_equal(E, ref.energy())
    rpar, rcnt = ref.parents()
    rc = ref.ctl()
    for p in parts:
        np.testing.assert_array_equal(p["parent"], rpar)
        np.testing.assert_array_equal(p["count"], rcnt)
        np.testing.assert_array_equal(p["hist"], ref.history())
        for k in ("t", "z", "cycle", "cooldown", "enable_cm", "done", "ncm_last", "hist_len"):
            assert p["ctl"][k] == rc[k], k
        assert p["ctl"]["beta"] == rc["beta"] and p["ctl"]["delta"] == rc["delta"]
        np.testing.assert_array_equal(p["targets"], ref.ncm_targets())
        mstar, best = ref.best()
        assert p["cut"] == mstar
        np.testing.assert_array_equal(p["best"], best)
    # the cluster moves of each rank's own targets add up to the single run's
    assert sum(p["ctl"]["ncm_flipped"] for p in parts) == rc["ncm_flipped"]
    assert max(p["ctl"]["ncm_dE_max"] for p in parts) == rc["ncm_dE_max"] == 0
    if params.get("resample", 1):
        assert sum(p["moved"] for p in parts) > 0      # replicas did cross block edges
    else:
        assert sum(p["moved"] for p in parts) == 0     # independent chains never move
    if params.get("stagnation"):
        assert rc["cycle"] >= 1                        # a restart re-drew the population
        if params.get("kind", 0) == 0:
            assert rc["ncm_flipped"] > 0               # cluster moves ran (defined for Max-Cut only)
    ref.close()


def test_plan_routes_every_parent():
    """The exchange plan of every rank, for random parent maps (sorted, as
    systematic resampling makes them, and arbitrary): what rank q receives
    from rank r is exactly what r sends to q, in the same order, and every
    own slot's source row holds its parent."""
    import paper_2606_25203_gb300 as pg
    rng = np.random.default_rng(0)
    for R, G in ((16, 1), (16, 2), (32, 4), (96, 3), (256, 8)):
        for sort in (True, False):
            parent = rng.integers(0, R, size=R).astype(np.int32)
            if sort:
                parent.sort()
            plans = [pg.pamc_shard_plan(R, G, g, parent) for g in range(G)]
            c = R // G
            # what each rank sends, in global indices, per destination
            sent = {}
            for g, (sc, rows, rcv, lp) in enumerate(plans):
                assert sc[g] == 0 and rcv[g] == 0
                off = 0
                for q in range(G):
                    sent[(g, q)] = (g * c + rows[off:off + sc[q]]).tolist()
                    off += sc[q]
                assert off == len(rows)
            for q, (sc, rows, rcv, lp) in enumerate(plans):
                src = [None] * (c + int(rcv.sum()))
                for j in range(c):
                    src[j] = q * c + j
                k = c
                for g in range(G):
                    got = sent[(g, q)]
                    assert len(got) == rcv[g]
                    for x in got:
                        src[k] = x
                        k += 1
                for m in range(c):
                    assert src[lp[m]] == parent[q * c + m]
                # only distinct foreign parents are received
                own = parent[q * c:(q + 1) * c]
                foreign = set(own[(own < q * c) | (own >= (q + 1) * c)].tolist())
                assert int(rcv.sum()) == len(foreign)
    with pytest.raises(pg.PamcError):
        pg.pamc_shard_plan(16, 2, 0, np.full(16, 16, dtype=np.int32))
    with pytest.raises(pg.PamcError):
        pg.pamc_shard_range(20, 2, 0)     # 20 is not a multiple of 4 x 2
