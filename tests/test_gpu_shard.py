"""One population split over several library handles on one GPU: each handle
holds a block of the slots and the package's exchange (``run_step``) moves
the energies and migrating replicas between them, here through an
in-process communicator (one thread per handle; every handle runs on the
default stream, the exchange waits for the device before it hands data
over, and no kernel waits on another handle).  The split run must equal the
single-handle run (pamc_step) of the same population bit for bit -- spins,
energies, parents, counts, the controller, M* and its configuration -- and,
at the small size, the oracle.  Covers the byte-lane and 16-bit-lane Ising
sweeps, spin words in device memory, both Potts samplers, cluster moves and
restarts."""
import threading

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

CTL_KEYS = ("t", "z", "cycle", "cooldown", "enable_cm", "done", "ncm_last", "hist_len")


@pytest.fixture(scope="module")
def pg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_25203_gb300 as pg
    pg.load()
    return pg


class _Group:
    def __init__(self, size):
        self.size = size
        self.slots = [None] * size
        self.barrier = threading.Barrier(size, timeout=300)

    def exchange(self, rank, item):
        self.slots[rank] = item
        self.barrier.wait()
        items = list(self.slots)
        self.barrier.wait()
        return items


class ThreadComm:
    """all_gather / all_to_all / broadcast between threads of one process."""

    def __init__(self, group, rank):
        import torch
        self.torch = torch
        self.group, self.rank, self.size = group, rank, group.size

    def _share(self, t):
        x = None if t is None else t.clone()
        self.torch.cuda.synchronize()
        return self.group.exchange(self.rank, x)

    def all_gather(self, out, inp):
        items = self._share(inp)
        out.copy_(self.torch.cat(items))
        self.torch.cuda.synchronize()

    def all_to_all(self, recv, send, recv_splits, send_splits):
        x = send.clone()
        self.torch.cuda.synchronize()
        items = self.group.exchange(self.rank, (x, list(send_splits)))
        parts = []
        for q, (xq, sq) in enumerate(items):
            off = sum(sq[:self.rank])
            assert sq[self.rank] == recv_splits[q]
            parts.append(xq[off:off + sq[self.rank]])
        if recv.numel():
            recv.copy_(self.torch.cat(parts))
        self.torch.cuda.synchronize()

    def broadcast(self, t, src):
        items = self._share(t if self.rank == src else None)
        t.copy_(items[src])
        self.torch.cuda.synchronize()


def run_split(pg, inst, G, nsteps, params):
    from paper_2606_25203_gb300 import shard as S
    group = _Group(G)
    out, errs = [None] * G, []

    def work(rank):
        try:
            sh = S.LibShard(inst.row_ptr, inst.col, inst.w, rank, G, **params)
            comm = ThreadComm(group, rank)
            for _ in range(nsteps):
                S.run_step(sh, comm)
            cut, best = S.best(sh, comm)
            spins, E, par, cnt = pg.pamc_state(sh.h, sh.count, inst.n)
            out[rank] = dict(spins=spins, E=E, par=par, cnt=cnt, ctl=pg.pamc_control_state(sh.h),
                             hist=pg.pamc_control_history(sh.h), cut=cut, best=best, moved=sh.moved,
                             mode=pg.pamc_sweep_mode(sh.h) if params.get("kind", 0) == 0 else None)
            sh.close()
        except BaseException as e:   # noqa: BLE001 -- re-raised below
            errs.append(e)
            group.barrier.abort()

    threads = [threading.Thread(target=work, args=(r,)) for r in range(G)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errs:
        raise errs[0]
    return out


def run_single(pg, inst, nsteps, params):
    h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
    p = pg.pamc_init(h, **params)
    pg.pamc_step(h, nsteps)
    spins, E, par, cnt = pg.pamc_state(h, p.R, inst.n)
    res = dict(spins=spins, E=E, par=par, cnt=cnt, ctl=pg.pamc_control_state(h), hist=pg.pamc_control_history(h),
               best=pg.pamc_best(h, inst.n), mode=pg.pamc_sweep_mode(h) if params.get("kind", 0) == 0 else None)
    pg.pamc_destroy(h)
    return res


def assert_split_equals(parts, ref, where):
    np.testing.assert_array_equal(np.concatenate([p["spins"] for p in parts]), ref["spins"], err_msg=f"spins {where}")
    np.testing.assert_array_equal(np.concatenate([p["E"] for p in parts]), ref["E"], err_msg=f"energies {where}")
    np.testing.assert_array_equal(np.concatenate([p["par"] for p in parts]), ref["par"], err_msg=f"parents {where}")
    np.testing.assert_array_equal(np.concatenate([p["cnt"] for p in parts]), ref["cnt"], err_msg=f"counts {where}")
    for p in parts:
        for k in CTL_KEYS:
            assert p["ctl"][k] == ref["ctl"][k], f"{k} {where}"
        assert p["ctl"]["beta"] == ref["ctl"]["beta"] and p["ctl"]["delta"] == ref["ctl"]["delta"], where
        np.testing.assert_array_equal(p["hist"][0], ref["hist"][0], err_msg=f"history {where}")
        assert p["hist"][1] == ref["hist"][1], f"M* {where}"
        cut, best = ref["best"]
        assert p["cut"] == cut, f"M* {where}"
        np.testing.assert_array_equal(p["best"], best, err_msg=f"best {where}")
    assert sum(p["ctl"]["ncm_flipped"] for p in parts) == ref["ctl"]["ncm_flipped"], where


AUG = dict(sweeps=2, beta0=0.5, beta1=6.0, stagnation=1, z_rst=120, cooldown_tau=5, seed=3)


@pytest.mark.parametrize("G", [1, 2, 4])
def test_split_equals_single_and_oracle_small(pg, G):
    """Torus 14 x 14, R = 32, 150 augmented steps (resampling across the
    block edges, cluster moves, reheats, a restart): the split run, the
    single-handle run and the oracle agree."""
    inst = W.torus(14, 14, signed=True, seed=2)
    steps = 150
    params = dict(R=32, steps=steps, **AUG)
    parts = run_split(pg, inst, G, steps, params)
    ref = run_single(pg, inst, steps, params)
    assert_split_equals(parts, ref, f"G={G}")
    orc = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, R=32, steps=steps, **AUG)
    orc.step(steps)
    np.testing.assert_array_equal(ref["spins"], orc.spins())
    assert ref["best"][0] == orc.best()[0]
    assert orc.ctl()["ncm_flipped"] > 0 and orc.ctl()["cycle"] >= 1
    if G > 1:
        assert sum(p["moved"] for p in parts) > 0
    orc.close()


@pytest.mark.parametrize("case", ["sparse_ncm", "potts_cascaded", "potts_softmax", "wide_lanes", "global_words",
                                  "large_population"])
def test_split_equals_single_handle(pg, monkeypatch, case):
    G = 4
    if case == "sparse_ncm":
        inst = W.c2b_sparse7000()
        params = dict(R=512, steps=60, sweeps=3, beta0=0.1, beta1=3.0, stagnation=1, win_short=2, win_long=3,
                      z_rst=45, cooldown_tau=3, seed=11)
    elif case == "potts_cascaded":
        inst = W.gnm(600, 3000, signed=False, seed=4)
        params = dict(kind=1, R=64, steps=40, sweeps=2, beta0=0.1, beta1=3.0, z_rst=30, seed=5)
    elif case == "potts_softmax":
        inst = W.gnm(400, 1600, signed=True, seed=6)
        params = dict(kind=1, rule=2, K=5, gamma=0.3, R=32, steps=30, sweeps=2, beta0=0.1, beta1=3.0, seed=7)
    elif case == "wide_lanes":
        from test_gpu_parity import _weighted_hub
        inst = _weighted_hub()
        params = dict(R=64, steps=40, sweeps=2, beta0=0.01, beta1=0.5, stagnation=1, z_rst=30, seed=8)
    elif case == "large_population":   # 32,768 replicas: the population step in several kernels
        inst = W.torus(10, 10, signed=True, seed=2)
        params = dict(R=32768, steps=12, sweeps=2, beta0=0.3, beta1=3.0, stagnation=1, win_short=2, win_long=3,
                      cooldown_tau=1, z_rst=9, seed=12)
    else:
        monkeypatch.setenv("PAMC_SWEEP_GLOBAL", "1")
        inst = W.torus(40, 40, signed=True, seed=1)
        params = dict(R=128, steps=40, sweeps=2, beta0=0.2, beta1=3.0, stagnation=1, z_rst=30, seed=9)
    parts = run_split(pg, inst, G, params["steps"], params)
    ref = run_single(pg, inst, params["steps"], params)
    assert_split_equals(parts, ref, case)
    assert all(p["mode"] == ref["mode"] for p in parts)
    if case == "wide_lanes":
        assert ref["mode"] & 8
    if case == "global_words":
        assert ref["mode"] & 4
    assert sum(p["moved"] for p in parts) > 0


def _run_split_dense(pg, w, G, nsteps, params):
    from paper_2606_25203_gb300 import shard as S
    group = _Group(G)
    out, errs = [None] * G, []

    def work(rank):
        try:
            sh = S.LibShard(None, None, None, rank, G, dense_w=w, **params)
            comm = ThreadComm(group, rank)
            for _ in range(nsteps):
                S.run_step(sh, comm)
            cut, best = S.best(sh, comm)
            spins, E, par, cnt = pg.pamc_state(sh.h, sh.count, sh.n)
            out[rank] = dict(spins=spins, E=E, par=par, cnt=cnt, ctl=pg.pamc_control_state(sh.h),
                             hist=pg.pamc_control_history(sh.h), cut=cut, best=best, moved=sh.moved)
            sh.close()
        except BaseException as e:   # noqa: BLE001 -- re-raised below
            errs.append(e)
            group.barrier.abort()

    threads = [threading.Thread(target=work, args=(r,)) for r in range(G)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errs:
        raise errs[0]
    return out


@pytest.mark.parametrize("G", [2, 4])
def test_split_dense_equals_single_handle(pg, G):
    """A dense +-1 instance (n = 2,048) with R = 64 split over two and four
    handles (the dense sweep's chains and tensor-core field updates on each
    handle's replicas, draws keyed by the global replica index) equals the
    single-handle run, through a restart that re-draws the population."""
    n = 2048
    w = W.dense_rows_np(n, np.arange(n), seed=4)
    params = dict(R=64, steps=30, sweeps=2, beta0=0.05, beta1=1.5, z_rst=17, seed=21)
    parts = _run_split_dense(pg, w, G, params["steps"], params)
    h = pg.pamc_create_dense(n, w)
    p = pg.pamc_init(h, **params)
    pg.pamc_step(h, params["steps"])
    spins, E, par, cnt = pg.pamc_state(h, p.R, n)
    ref = dict(spins=spins, E=E, par=par, cnt=cnt, ctl=pg.pamc_control_state(h), hist=pg.pamc_control_history(h),
               best=pg.pamc_best(h, n))
    pg.pamc_destroy(h)
    assert_split_equals(parts, ref, f"dense G={G}")
    assert ref["ctl"]["cycle"] >= 1
    assert sum(p["moved"] for p in parts) > 0


def test_split_phase_order_and_refusals(pg):
    """Calls out of order and the single-population calls on a split handle
    are refused on the host; a bad plan argument is refused before any
    device work."""
    import torch
    inst = W.torus(8, 8, signed=True, seed=0)
    h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
    with pytest.raises(pg.PamcError):
        pg.pamc_shard_init(h, 0, 2, R=30, steps=5)            # 30 is not a multiple of 4 x 2
    pg.pamc_shard_init(h, 1, 2, R=16, steps=5, sweeps=1)
    E_all = torch.zeros(16, dtype=torch.int64, device="cuda")
    E_own = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(pg.PamcError) as e:
        pg.pamc_shard_sweep(h, E_all, np.zeros(8, dtype=np.int32), None, 0, E_own)
    assert e.value.status == pg.STATUS_CODES["PAMC_ERR_STATE"]
    with pytest.raises(pg.PamcError) as e:
        pg.pamc_step(h, 1)
    assert e.value.status == pg.STATUS_CODES["PAMC_ERR_STATE"]
    pg.pamc_shard_energies(h, E_own)
    E_all[8:] = E_own
    E_all[:8] = E_own
    parent = pg.pamc_shard_resample(h, E_all)
    assert np.array_equal(parent, np.arange(16))             # the first iteration keeps the population
    with pytest.raises(pg.PamcError) as e:                    # a source row past the received ones
        pg.pamc_shard_sweep(h, E_all, np.full(8, 8, dtype=np.int32), None, 0, E_own)
    assert e.value.status == pg.STATUS_CODES["PAMC_ERR_RANGE"]
    with pytest.raises(pg.PamcError):
        pg.pamc_shard_pack(h, np.array([8], dtype=np.int32), torch.zeros(inst.n, dtype=torch.int8, device="cuda"))
    pg.pamc_shard_sweep(h, E_all, np.arange(8, dtype=np.int32), None, 0, E_own)
    pg.pamc_shard_control(h, E_all, E_own)
    pg.pamc_sync(h)
    with pytest.raises(pg.PamcError):
        pg.pamc_hamming(h, inst.n)
    pg.pamc_destroy(h)
