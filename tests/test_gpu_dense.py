"""Dense (fully connected) instances through pamc_create_dense, compared with
the oracle on the same instance given as CSR.  Exact comparison of spins,
energies, resampling, controller state and best cut after every step."""
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


def dense_pair(n, seed):
    Jg = W.dense_rows_np(n, np.arange(n), seed)          # couplings, zero diagonal
    w = (-Jg).astype(np.int8)                             # Max-Cut weights
    return w, W.dense_csr(n, seed)


def compare_dense(pg, n, steps, seed=0, check_every=1, **params):
    w, inst = dense_pair(n, seed)
    ref = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, steps=steps, **params)
    h = pg.pamc_create_dense(n, w)
    try:
        p = pg.pamc_init(h, steps=steps, **params)
        R = p.R
        assert pg.pamc_weight_sum(h) == ref.weight_sum()
        done = 0
        while done < steps:
            k = min(check_every, steps - done)
            pg.pamc_step(h, k)
            ref.step(k)
            done += k
            spins, E, par, cnt = pg.pamc_state(h, R, n)
            where = f"after {done} steps"
            np.testing.assert_array_equal(spins, ref.spins(), err_msg=f"spins {where}")
            np.testing.assert_array_equal(E, ref.energy(), err_msg=f"energies {where}")
            rp, rc = ref.parents()
            np.testing.assert_array_equal(par, rp, err_msg=f"parents {where}")
            np.testing.assert_array_equal(cnt, rc, err_msg=f"counts {where}")
            gc, oc = pg.pamc_control_state(h), ref.ctl()
            for key in ("t", "z", "cycle", "cooldown", "enable_cm", "done"):
                assert gc[key] == oc[key], f"{key} {where}"
            assert gc["beta"] == oc["beta"] and gc["delta"] == oc["delta"], where
            m, b = pg.pamc_best(h, n)
            rm, rb = ref.best()
            assert m == rm, where
            np.testing.assert_array_equal(b, rb, err_msg=f"best {where}")
    finally:
        pg.pamc_destroy(h)


@pytest.mark.parametrize("rule", [0, 1])
def test_dense_small(pg, rule):
    compare_dense(pg, 256, 8, R=8, sweeps=2, beta0=0.01, beta1=0.3, rule=rule, seed=3)


def test_dense_ragged_n_and_population(pg):
    # n not a multiple of 16 (byte-copy path of the recompute), R not a
    # multiple of 4, several position blocks per sweep
    compare_dense(pg, 1000, 5, R=13, sweeps=2, beta0=0.02, beta1=0.5, seed=1)


def test_dense_full_population_multi_block(pg):
    compare_dense(pg, 2048, 4, R=64, sweeps=2, beta0=0.01, beta1=1.0, seed=2)


def test_dense_restart_and_controller(pg):
    compare_dense(pg, 320, 60, R=16, sweeps=1, beta0=0.01, beta1=0.4, stagnation=1, z_rst=45, seed=5,
                  check_every=3)


def test_dense_rejects(pg):
    n = 64
    w, _ = dense_pair(n, 0)
    bad = w.copy()
    bad[3, 5] = -bad[3, 5]                  # asymmetric
    with pytest.raises(pg.PamcError) as e:
        pg.pamc_create_dense(n, bad)
    assert e.value.status == 2
    bad = w.copy()
    bad[4, 4] = 1                            # diagonal
    with pytest.raises(pg.PamcError) as e:
        pg.pamc_create_dense(n, bad)
    assert e.value.status == 3
    h = pg.pamc_create_dense(n, w)
    with pytest.raises(pg.PamcError):
        pg.pamc_init(h, R=65, steps=2)       # more replicas than the chain masks hold
    pg.pamc_destroy(h)
    odd, _ = dense_pair(63, 0)
    h = pg.pamc_create_dense(63, odd)
    with pytest.raises(pg.PamcError):
        pg.pamc_init(h, R=8, steps=2, stagnation=1)
    pg.pamc_destroy(h)
