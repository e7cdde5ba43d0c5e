"""Step-replay parity at full size (Eq. 1-4, Algorithm 1).

The CUDA path runs a full-size population to a late step t.  Its whole state
(population, step index, controller, M* history, best cut and configuration)
is loaded into the oracle, and both compute iteration t -> t+1.  The oracle
resamples, picks and moves the cluster-move targets, runs M*, the best
configuration and the controller on the whole population; it sweeps a sample
of the replicas itself (random slots and cluster-move targets) and takes the
CUDA path's post-sweep configurations for the others, recomputing their
fields and energies from the definition.  Everything is compared exactly:
parents and copy counts of every slot, every energy, every spin, the
controller fields bit for bit, the history, M* and the best configuration.

Steps checked: a mid-anneal step, the first step that applies cluster moves
(the (energy, slot) target sort at R = 4,096 and the MIS kernel on the full
instance), and the restart that re-draws the population -- on the torus
141x141 and the sparse N=7,000 instance at R = 4,096 (the benchmark's
configuration), a late step of Max-3-Cut at R = 2,048, and a sparse instance
with n = 40,000 (schedules built with keys and counters in global memory).
The dense n = 100,000 instance is checked over a whole late step for sampled
replicas by a sequential replay of both sweeps from exact fields.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

CTL_EXACT = ("t", "z", "cycle", "cooldown", "enable_cm", "done", "ncm_last", "hist_len")


@pytest.fixture(scope="module")
def pg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_25203_gb300 as pg
    pg.load()
    return pg


def _gpu_state(pg, s):
    spins, E, par, cnt = s.state()
    hist, mstar = pg.pamc_control_history(s.h)
    m, best = s.best()
    assert m == mstar
    return dict(spins=spins, E=E, par=par, cnt=cnt, ctl=s.control(), hist=hist, mstar=mstar, best=best)


def _advance_to(pg, s, stop, limit):
    """Step the CUDA run one iteration at a time until stop(ctl) holds for the
    iteration about to run, at most up to step index limit."""
    while True:
        c = s.control()
        if stop(c) or c["t"] >= limit:
            return c
        s.step(1)


def _replay_one(pg, s, ref, rng, n_random=40, n_targets=12, want_ncm=None, want_restart=None):
    """Check iteration t -> t+1 of the CUDA run s against the oracle ref (same
    instance and parameters).  Returns the oracle's control fields after it."""
    a = _gpu_state(pg, s)
    s.step(1)
    b = _gpu_state(pg, s)
    R = a["spins"].shape[0]
    t = a["ctl"]["t"]

    def load():
        ref.set_state(t, a["ctl"], a["hist"], a["mstar"], a["best"], a["spins"])

    # pass 1: no sweeps of its own, to learn the cluster-move targets
    load()
    ref.set_sweep_replay(np.zeros(R, dtype=bool), b["spins"])
    ref.step(1)
    targets = ref.ncm_targets()
    # pass 2: random slots and some targets swept by the oracle
    mask = np.zeros(R, dtype=bool)
    mask[rng.choice(R, size=min(n_random, R), replace=False)] = True
    if targets.size:
        mask[targets[:n_targets]] = True
        mask[targets[-n_targets:]] = True
    load()
    ref.set_sweep_replay(mask, b["spins"])
    ref.step(1)
    where = f"step {t} -> {t + 1}"
    np.testing.assert_array_equal(b["spins"], ref.spins(), err_msg=f"spins {where}")
    np.testing.assert_array_equal(b["E"], ref.energy(), err_msg=f"energies {where}")
    rp, rc = ref.parents()
    np.testing.assert_array_equal(b["par"], rp, err_msg=f"parents {where}")
    np.testing.assert_array_equal(b["cnt"], rc, err_msg=f"counts {where}")
    oc = ref.ctl()
    for key in CTL_EXACT:
        assert b["ctl"][key] == oc[key], f"{key} {where}: {b['ctl'][key]} != {oc[key]}"
    assert b["ctl"]["beta"] == oc["beta"] and b["ctl"]["delta"] == oc["delta"], where
    assert b["ctl"]["ncm_flipped"] - a["ctl"]["ncm_flipped"] == oc["ncm_flipped"], where
    assert oc["ncm_dE_max"] == 0 and b["ctl"]["ncm_dE_max"] == 0, where
    np.testing.assert_array_equal(b["hist"], ref.history(), err_msg=f"history {where}")
    m, best = ref.best()
    assert b["mstar"] == m, where
    np.testing.assert_array_equal(b["best"], best, err_msg=f"best {where}")
    if want_ncm is not None:
        assert bool(oc["ncm_last"]) == want_ncm and (targets.size > 0) == want_ncm, where
    if want_restart is not None:
        assert (oc["cycle"] > a["ctl"]["cycle"]) == want_restart, where
    ref.set_sweep_replay()
    return oc, int(mask.sum()), int(targets.size)


C2 = dict(R=4096, sweeps=10, steps=500, beta0=0.1, beta1=4.0, stagnation=1, z_rst=400, seed=0)


@pytest.mark.parametrize("name", ["torus141", "sparse7000"])
def test_c2_full_size_replay_mid_ncm_restart(pg, name):
    """Configuration 2 at R = 4,096 (the benchmark's launch configuration):
    step 45 (control active), the first iteration that applies cluster moves,
    and the restart at z = 400 that re-draws the population."""
    inst = W.c2a_torus141() if name == "torus141" else W.c2b_sparse7000()
    rng = np.random.default_rng(1)
    s = pg.Solver(inst.row_ptr, inst.col, inst.w)
    s.init(**C2)
    ref = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, steps=C2["steps"],
                           **{k: v for k, v in C2.items() if k != "steps"})
    try:
        _advance_to(pg, s, lambda c: c["t"] >= 45, 45)
        _replay_one(pg, s, ref, rng, want_ncm=False)
        # the next iteration applies cluster moves when the controller armed
        # them at the end of the last one and no cooldown runs
        c = _advance_to(pg, s, lambda c: c["enable_cm"] == 1 and c["cooldown"] == 0, 398)
        assert c["enable_cm"] == 1 and c["cooldown"] == 0, "no stagnation before the restart"
        oc, _, ntg = _replay_one(pg, s, ref, rng, want_ncm=True)
        assert ntg == C2["R"] // 16 and oc["ncm_flipped"] > 0
        _advance_to(pg, s, lambda c: c["z"] >= C2["z_rst"], 420)
        _replay_one(pg, s, ref, rng, want_restart=True)
        _replay_one(pg, s, ref, rng, want_restart=False)   # first step of the new cycle
    finally:
        s.close()
        ref.close()


@pytest.mark.parametrize("rule", [0, 2])
def test_c3_potts_late_step_replay(pg, rule):
    """Configuration 3 at full size (N = 2,000, average degree 12, R = 2,048,
    10 sweeps), iteration 150 -> 151: resampling with the half-energy
    weights of the Potts reading and the sweeps of sampled replicas, both
    samplers."""
    inst = W.c3_sparse2000()
    params = dict(kind=1, rule=rule, R=2048, sweeps=10, steps=300, beta0=0.1, beta1=3.0, seed=0)
    if rule == 2:
        params.update(K=3, gamma=1.0)
    rng = np.random.default_rng(2)
    s = pg.Solver(inst.row_ptr, inst.col, inst.w)
    s.init(**params)
    ref = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **params)
    try:
        s.step(150)
        oc, swept, _ = _replay_one(pg, s, ref, rng, n_random=48)
        assert swept == 48 and oc["t"] == 151
    finally:
        s.close()
        ref.close()


def test_sparse40000_global_schedule_replay(pg):
    """n = 40,000 (average degree 5.7, +-1): above 20,480 the schedule kernel
    keeps its keys and predecessor counters in global memory.  Augmented
    PAMC at R = 512: a mid-anneal step and, when the controller arms them
    within 300 steps, the first cluster-move step."""
    inst = W.gnm(40000, 114000, signed=True, seed=4)
    params = dict(R=512, sweeps=4, steps=300, beta0=0.1, beta1=4.0, stagnation=1, z_rst=0, seed=3)
    rng = np.random.default_rng(3)
    s = pg.Solver(inst.row_ptr, inst.col, inst.w)
    s.init(**params)
    ref = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **params)
    try:
        s.step(60)
        _replay_one(pg, s, ref, rng, n_random=24, want_ncm=False)
        c = _advance_to(pg, s, lambda c: c["enable_cm"] == 1 and c["cooldown"] == 0, 298)
        if c["enable_cm"] == 1 and c["cooldown"] == 0:
            _replay_one(pg, s, ref, rng, n_random=16, n_targets=8, want_ncm=True)
    finally:
        s.close()
        ref.close()


def test_dense100k_whole_late_step_replay(pg):
    """Configuration 4's instance and population (n = 100,000, R = 64,
    2 sweeps, beta 0.01 -> 1.0 over 200 steps) at iteration 100 -> 101:
    parents and counts of every slot against the oracle's resampling of the
    energies; for sampled slots both whole sweeps (200,000 positions) are
    replayed sequentially on the CPU from exact fields (an fp32 product of J
    and the parent's configuration on CUDA cores, exact below 2^24), with
    the oracle's order, draws and thresholds; every spin and the energy of
    those slots must match."""
    import torch
    n, R, seed = 100000, 64, 0
    params = dict(R=R, sweeps=2, steps=200, beta0=0.01, beta1=1.0, seed=0)
    t0 = 100
    wd = torch.empty((n, n), dtype=torch.int8, device="cuda")
    for r0 in range(0, n, 2000):
        wd[r0:r0 + 2000] = -W.dense_rows_torch(n, r0, min(n, r0 + 2000), seed, device="cuda")
    h = pg.pamc_create_dense(n, wd)
    Jd = wd.neg_()                       # J = -w, on the device for the exact fields
    try:
        pg.pamc_init(h, **params)
        pg.pamc_step(h, t0)
        S0, E0, _, _ = pg.pamc_state(h, R, n)
        c0 = pg.pamc_control_state(h)
        assert c0["t"] == t0
        pg.pamc_step(h, 1)
        S1, E1, par, cnt = pg.pamc_state(h, R, n)
        c1 = pg.pamc_control_state(h)
    finally:
        pg.pamc_destroy(h)
    rpar, rcnt = oracle.resample(E0, c0["delta"], 1.0, params["seed"], t0)
    np.testing.assert_array_equal(par, rpar)
    np.testing.assert_array_equal(cnt, rcnt)
    assert c1["beta"] == c0["beta"] + c0["delta"]
    beta = c0["beta"]
    rng = np.random.default_rng(4)
    slots = np.sort(rng.choice(R, size=6, replace=False))
    X = S0[par[slots]].astype(np.int8)                       # configurations entering the sweeps
    Sf = torch.from_numpy(X).cuda().float().T.contiguous()
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        hcur = torch.empty((n, len(slots)), dtype=torch.int64, device="cuda")
        for r0 in range(0, n, 4096):
            hcur[r0:r0 + 4096] = (Jd[r0:r0 + 4096].float() @ Sf).round().long()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    hcur = hcur.cpu().numpy().T.copy()                       # slots x n
    del Jd, wd
    torch.cuda.empty_cache()
    s = X.astype(np.int64)
    E = E0[par[slots]].astype(np.int64).copy()
    key = (params["seed"] & 0xFFFFFFFF, params["seed"] >> 32)
    thr = {}
    rows = {}
    groups = sorted({int(r) // 4 for r in slots})
    for sw in range(params["sweeps"]):
        order = oracle.permutation(n, params["seed"], t0, sw)
        for k in order.tolist():
            u = {g: oracle.philox4x32_10((k, sw, t0, (oracle.TAG_FLIP << 24) | g), key) for g in groups}
            for i, r in enumerate(slots.tolist()):
                hv = int(hcur[i, k])
                if hv not in thr:
                    thr[hv] = oracle.thr_heatbath(beta, hv)
                new = 1 if int(u[r // 4][r % 4]) < thr[hv] else -1
                if new != s[i, k]:
                    E[i] += 2 * s[i, k] * hv
                    s[i, k] = new
                    if k not in rows:
                        rows[k] = W.dense_rows_np(n, np.array([k]), seed)[0].astype(np.int64)
                    hcur[i] += 2 * new * rows[k]
    np.testing.assert_array_equal(S1[slots], s.astype(np.int8))
    np.testing.assert_array_equal(E1[slots], E)
    assert len(rows) > 0                                      # flips happened in the replayed step


def test_sparse80000_device_memory_spins_replay(pg):
    """n = 80,000 (average degree 5.7, +-1): a replica group's spin words
    (320 KB) no longer fit shared memory, so they live in device memory.
    Augmented PAMC at R = 64: iterations 10 -> 11 and 30 -> 31 replayed."""
    inst = W.gnm(80000, 228000, signed=True, seed=6)
    params = dict(R=64, sweeps=2, steps=100, beta0=0.1, beta1=4.0, stagnation=1, z_rst=0, seed=5)
    rng = np.random.default_rng(6)
    s = pg.Solver(inst.row_ptr, inst.col, inst.w)
    s.init(**params)
    assert pg.pamc_sweep_mode(s.h) & 4
    ref = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **params)
    try:
        s.step(10)
        _replay_one(pg, s, ref, rng, n_random=12)
        s.step(19)
        _replay_one(pg, s, ref, rng, n_random=12)
    finally:
        s.close()
        ref.close()
