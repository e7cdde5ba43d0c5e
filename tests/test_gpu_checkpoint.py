"""Checkpoints (pamc_save / pamc_load): a run saved at step t and continued
on a fresh handle of the same instance is the uninterrupted run, bit for bit
-- spins, energies, parents, counts, the controller and its M* history, M*
and its configuration, the lineage -- through resampling, cluster moves,
reheats and a restart, for Max-Cut, Max-3-Cut and a dense instance; the
uninterrupted run itself equals the oracle.  Checkpoints of another
instance, truncated ones and corrupted ones are refused on the host."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_25203_gb300 as pg
    pg.load()
    return pg


def _full_state(pg, s):
    spins, E, par, cnt = s.state()
    fam, nf = pg.pamc_lineage(s.h, s.R)
    return dict(spins=spins, E=E, par=par, cnt=cnt, ctl=s.control(), hist=pg.pamc_control_history(s.h),
                best=s.best(), fam=fam, nf=nf)


def _same(a, b):
    for k in ("spins", "E", "par", "cnt", "fam"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    assert a["ctl"] == b["ctl"]
    np.testing.assert_array_equal(a["hist"][0], b["hist"][0])
    assert a["hist"][1] == b["hist"][1]
    assert a["best"][0] == b["best"][0] and a["nf"] == b["nf"]
    np.testing.assert_array_equal(a["best"][1], b["best"][1])


CASES = {
    "maxcut_augmented": (lambda: W.torus(16, 16, signed=True, seed=1),
                         dict(R=40, sweeps=2, steps=150, beta0=0.5, beta1=6.0, stagnation=1, z_rst=100,
                              cooldown_tau=5, seed=3), 70),
    "max3cut": (lambda: W.gnm(300, 1500, signed=False, seed=4),
                dict(kind=1, R=24, sweeps=2, steps=60, beta0=0.1, beta1=3.0, z_rst=40, seed=5), 25),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_resume_equals_uninterrupted_run(pg, case):
    make, params, t_save = CASES[case]
    inst = make()
    steps = params["steps"]
    full = pg.Solver(inst.row_ptr, inst.col, inst.w)
    full.init(**params)
    full.step(t_save)
    ckpt = full.save()
    full.step(steps - t_save)
    ref = _full_state(pg, full)
    # a fresh handle of the same instance, loaded from the checkpoint
    res = pg.Solver(inst.row_ptr, inst.col, inst.w)
    res.load(ckpt, params["R"])
    assert res.control()["t"] == t_save
    res.step(steps - t_save)
    _same(_full_state(pg, res), ref)
    # loading twice from the same bytes gives the same run again
    res.load(ckpt, params["R"])
    res.step(steps - t_save)
    _same(_full_state(pg, res), ref)
    orc = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **params)
    orc.step(steps)
    np.testing.assert_array_equal(ref["spins"], orc.spins())
    assert ref["best"][0] == orc.best()[0]
    if case == "maxcut_augmented":
        assert orc.ctl()["ncm_flipped"] > 0 and orc.ctl()["cycle"] >= 1
    for s in (full, res):
        s.close()
    orc.close()


def test_dense_resume(pg):
    n = 256
    w = W.dense_rows_np(n, np.arange(n), seed=2)
    params = dict(R=16, sweeps=2, steps=40, beta0=0.05, beta1=1.5, z_rst=30, seed=6)
    a = pg.pamc_create_dense(n, w)
    pg.pamc_init(a, **params)
    pg.pamc_step(a, 12)
    ckpt = pg.pamc_save(a)
    pg.pamc_step(a, 28)
    ref = pg.pamc_state(a, 16, n), pg.pamc_best(a, n), pg.pamc_control_state(a)
    b = pg.pamc_create_dense(n, w)
    pg.pamc_load(b, ckpt)
    pg.pamc_step(b, 28)
    got = pg.pamc_state(b, 16, n), pg.pamc_best(b, n), pg.pamc_control_state(b)
    for x, y in zip(ref[0], got[0]):
        np.testing.assert_array_equal(x, y)
    assert ref[1][0] == got[1][0]
    np.testing.assert_array_equal(ref[1][1], got[1][1])
    assert ref[2] == got[2]
    pg.pamc_destroy(a)
    pg.pamc_destroy(b)


def test_bad_checkpoints_are_refused(pg):
    inst = W.torus(8, 8, signed=True, seed=0)
    other = W.torus(8, 8, signed=True, seed=1)      # same size, other weights
    s = pg.Solver(inst.row_ptr, inst.col, inst.w)
    s.init(R=8, sweeps=1, steps=10, seed=1)
    s.step(3)
    ck = s.save()
    t = pg.Solver(other.row_ptr, other.col, other.w)
    with pytest.raises(pg.PamcError) as e:
        t.load(ck, 8)
    assert e.value.status == pg.STATUS_CODES["PAMC_ERR_ARG"]
    with pytest.raises(pg.PamcError) as e:
        s.load(ck[:-1], 8)
    assert e.value.status == pg.STATUS_CODES["PAMC_ERR_ARG"]
    bad = bytearray(ck)
    # the first spin of the population (after the header and the controller)
    # set to a value no Max-Cut spin takes
    spin0 = len(ck) - (8 * 64 + 8 * 8 + 8 * 16 + 64)
    bad[spin0] = 5
    with pytest.raises(pg.PamcError) as e:
        s.load(bytes(bad), 8)
    assert e.value.status == pg.STATUS_CODES["PAMC_ERR_RANGE"]
    # the refusals left the run as it was
    s.load(ck, 8)
    assert s.control()["t"] == 3
    s.close()
    t.close()
