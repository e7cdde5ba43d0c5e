"""The oracle's step replay (orc_set_state, orc_set_sweep_replay) against the
oracle's own uninterrupted runs, on the CPU.

The GPU parity tests at full population size load a state the CUDA path
reached into the oracle and let it compute the next iteration with the sweeps
of a sample of replicas (the others take the CUDA path's results).  Here the
same machinery is checked against the oracle itself: a run resumed from its
own state at step t is the same run, and an iteration with sampled sweeps
whose other replicas take the full run's results equals the full iteration in
every spin, energy, parent, count, controller field and best cut.  Runs cover
resampling, cluster moves, reheats and a restart."""
import numpy as np
import pytest

import oracle
import workloads as W


def _snapshot(run):
    return dict(t=run.ctl()["t"], ctl=run.ctl(), hist=run.history(), best=run.best(), spins=run.spins())


def _load(run, snap):
    m, b = snap["best"]
    run.set_state(snap["t"], snap["ctl"], snap["hist"], m, b, snap["spins"])


def _assert_same(a, b, where):
    np.testing.assert_array_equal(a.spins(), b.spins(), err_msg=f"spins {where}")
    np.testing.assert_array_equal(a.energy(), b.energy(), err_msg=f"energies {where}")
    pa, ca = a.parents()
    pb, cb = b.parents()
    np.testing.assert_array_equal(pa, pb, err_msg=f"parents {where}")
    np.testing.assert_array_equal(ca, cb, err_msg=f"counts {where}")
    ka, kb = a.ctl(), b.ctl()
    for key in ("t", "z", "cycle", "cooldown", "enable_cm", "done", "ncm_last", "hist_len"):
        assert ka[key] == kb[key], f"{key} {where}"
    assert ka["beta"] == kb["beta"] and ka["delta"] == kb["delta"], where
    np.testing.assert_array_equal(a.history(), b.history(), err_msg=f"history {where}")
    ma, ba = a.best()
    mb, bb = b.best()
    assert ma == mb, f"M* {where}"
    np.testing.assert_array_equal(ba, bb, err_msg=f"best {where}")


PARAMS = [dict(R=24, sweeps=2, steps=150, beta0=0.5, beta1=6.0, stagnation=1, z_rst=120, cooldown_tau=5, seed=3),
          dict(kind=1, R=12, sweeps=2, steps=90, beta0=0.5, beta1=5.0, stagnation=1, z_rst=70, cooldown_tau=4,
               seed=4)]


@pytest.mark.parametrize("params", PARAMS, ids=["ising_ncm", "potts"])
def test_resume_from_own_state_is_the_same_run(params):
    inst = W.torus(14, 14, signed=True, seed=2)
    full = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **params)
    for t0 in (0, 37, 61, 118):
        full.step(t0 - full.ctl()["t"])
        snap = _snapshot(full)
        resumed = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **params)
        _load(resumed, snap)
        for k in range(6):
            full.step(1)
            resumed.step(1)
            ref_k = full.ctl()
            _assert_same(full, resumed, f"t0={t0} +{k + 1}")
            assert resumed.ctl()["ncm_flipped"] == ref_k["ncm_flipped"] - snap["ctl"]["ncm_flipped"]
        resumed.close()
        # rewind the full run's own counters to compare the next window
    full.close()


def test_sampled_sweeps_equal_the_full_iteration():
    """Every step of an augmented run (resampling, NCM, reheats, a restart)
    replayed with a random half of the replicas swept and the rest taken
    from the full run's result: identical to the full iteration."""
    inst = W.torus(14, 14, signed=True, seed=2)
    params = PARAMS[0]
    full = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **params)
    rep = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **params)
    rng = np.random.default_rng(5)
    saw_ncm = saw_restart = 0
    for step in range(params["steps"]):
        snap = _snapshot(full)
        full.step(1)
        _load(rep, snap)
        mask = rng.random(params["R"]) < 0.5
        rep.set_sweep_replay(mask, full.spins())
        rep.step(1)
        _assert_same(full, rep, f"step {step}")
        if full.ctl()["ncm_last"]:
            saw_ncm += 1
            assert len(rep.ncm_targets()) == max(1, params["R"] // 16)
        saw_restart = max(saw_restart, full.ctl()["cycle"])
    assert saw_ncm > 0 and saw_restart == 1
    full.close()
    rep.close()


def test_sampled_sweeps_detect_a_wrong_sample():
    """A replica of the sample is swept by the oracle itself: handing it a
    wrong configuration changes nothing, while handing a wrong configuration
    to a replica outside the sample is taken as given (so the comparison with
    the other path would fail there)."""
    inst = W.torus(10, 10, signed=True, seed=1)
    params = dict(R=8, sweeps=2, steps=20, beta0=0.5, beta1=3.0, seed=2)
    full = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **params)
    full.step(5)
    snap = _snapshot(full)
    full.step(1)
    after = full.spins()
    bad = after.copy()
    bad[[1, 6]] = -bad[[1, 6]]
    rep = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **params)
    _load(rep, snap)
    mask = np.zeros(8, dtype=bool)
    mask[1] = True
    rep.set_sweep_replay(mask, bad)
    rep.step(1)
    got = rep.spins()
    np.testing.assert_array_equal(got[1], after[1])      # swept by the oracle
    np.testing.assert_array_equal(got[6], bad[6])        # taken as given
    rep.close()
    full.close()


def test_sweep_flip_count_is_the_number_of_changed_spins():
    """With one sweep per step and no resampling, a spin changes at most once
    per step at its one visit, so the flips of a step are the spins that
    differ before and after it."""
    inst = W.torus(12, 12, signed=True, seed=3)
    run = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, R=8, sweeps=1, steps=12, resample=0, seed=1)
    total = 0
    prev = run.spins()
    for _ in range(12):
        run.step(1)
        cur = run.spins()
        total += int((cur != prev).sum())
        prev = cur
        assert run.sweep_flips() == total
    run.close()
