"""pamc_sweeps_noalloc: S sweeps at a fixed beta for callers that cannot
allocate device memory (they may only use the buffers they are handed, e.g.
a plug-in inside a framework that owns all device memory).  Its output must
equal what the regular entry points compute: pamc_step on the same population
at the same step index, with resampling off so that a step is exactly S
sweeps at the current beta.  Two calls in a row, exact comparison (spins and
integer energies).  This file is collected last on purpose."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_25203_gb300 as pg
    pg.load()
    return pg, torch


def _dev_csr(torch, inst):
    rp = torch.from_numpy(inst.row_ptr.astype(np.int32)).cuda()
    col = torch.from_numpy(inst.col.astype(np.int32)).cuda()
    w = torch.from_numpy(inst.w.astype(np.int32)).cuda()
    H = int(max(np.abs(inst.w[inst.row_ptr[i]:inst.row_ptr[i + 1]]).sum()
                for i in range(inst.n)))
    return rp, col, w, H


@pytest.mark.parametrize("rule", [0, 1])
@pytest.mark.parametrize("which", ["torus", "sparse"])
def test_noalloc_matches_pamc_step_twice(env, rule, which):
    pg, torch = env
    inst = W.torus(20, 20, signed=True, seed=3) if which == "torus" else W.gnm(1500, 4000, seed=5)
    R, S, steps, b0, b1, seed = 13, 3, 5, 0.3, 2.0, 9
    s = pg.Solver(inst.row_ptr, inst.col, inst.w)
    s.init(R=R, sweeps=S, steps=steps, beta0=b0, beta1=b1, resample=0, rule=rule, seed=seed)
    spins0, _, _, _ = s.state()
    rp, col, w, H = _dev_csr(torch, inst)
    x = torch.from_numpy(spins0).cuda()
    y = torch.empty_like(x)
    E = torch.empty(R, dtype=torch.int64, device="cuda")
    beta = b0
    dbeta = (b1 - b0) / (steps - 1)
    for t in (0, 1):
        pg.pamc_sweeps_noalloc(inst.n, inst.nnz, rp, col, w, H, rule, R, S, beta, seed, t, x, y, E)
        s.step(1)
        spins, Eref, _, _ = s.state()
        np.testing.assert_array_equal(y.cpu().numpy(), spins)
        np.testing.assert_array_equal(E.cpu().numpy(), Eref)
        x, y = y, x
        beta = beta + dbeta
    s.close()


def test_noalloc_in_place_and_limits(env):
    pg, torch = env
    inst = W.gnm(500, 1200, seed=2)
    R, S, seed = 8, 2, 4
    s = pg.Solver(inst.row_ptr, inst.col, inst.w)
    s.init(R=R, sweeps=S, steps=3, beta0=0.5, beta1=1.5, resample=0, seed=seed)
    spins0, _, _, _ = s.state()
    rp, col, w, H = _dev_csr(torch, inst)
    x = torch.from_numpy(spins0).cuda()
    E = torch.empty(R, dtype=torch.int64, device="cuda")
    pg.pamc_sweeps_noalloc(inst.n, inst.nnz, rp, col, w, H, 0, R, S, 0.5, seed, 0, x, x, E)
    s.step(1)
    spins, Eref, _, _ = s.state()
    np.testing.assert_array_equal(x.cpu().numpy(), spins)
    np.testing.assert_array_equal(E.cpu().numpy(), Eref)
    s.close()
    # sizes beyond the static scratch are rejected before any device work
    for kw in (dict(n=32769), dict(nnz=262145), dict(sweeps=9), dict(R=16385), dict(H=128)):
        a = dict(n=inst.n, nnz=inst.nnz, sweeps=S, R=R, H=H)
        a.update(kw)
        with pytest.raises(pg.PamcError) as ei:
            pg.pamc_sweeps_noalloc(a["n"], a["nnz"], rp, col, w, a["H"], 0, a["R"], a["sweeps"],
                                   0.5, seed, 0, x, x, E)
        assert ei.value.status == 4
    # an understated field bound is caught by the validation kernel
    with pytest.raises(pg.PamcError) as ei:
        pg.pamc_sweeps_noalloc(inst.n, inst.nnz, rp, col, w, 1, 0, R, S, 0.5, seed, 0, x, x, E)
    assert ei.value.status == 4


def test_noalloc_large_instance_global_schedule_path(env):
    """n = 25,000 (the schedule keeps its keys and counters in global memory
    above n = 20,480; eight warps per group) with nnz close to the scratch's
    limit, one sweep, a small population: equal to pamc_step, twice."""
    pg, torch = env
    inst = W.gnm(25000, 130000, seed=8)
    assert inst.nnz <= 262144
    R, S, steps, seed = 6, 1, 3, 2
    s = pg.Solver(inst.row_ptr, inst.col, inst.w)
    s.init(R=R, sweeps=S, steps=steps, beta0=0.4, beta1=1.2, resample=0, seed=seed)
    spins0, _, _, _ = s.state()
    rp, col, w, H = _dev_csr(torch, inst)
    x = torch.from_numpy(spins0).cuda()
    y = torch.empty_like(x)
    E = torch.empty(R, dtype=torch.int64, device="cuda")
    beta = 0.4
    for t in (0, 1):
        pg.pamc_sweeps_noalloc(inst.n, inst.nnz, rp, col, w, H, 0, R, S, beta, seed, t, x, y, E)
        s.step(1)
        spins, Eref, _, _ = s.state()
        np.testing.assert_array_equal(y.cpu().numpy(), spins)
        np.testing.assert_array_equal(E.cpu().numpy(), Eref)
        x, y = y, x
        beta = beta + (1.2 - 0.4) / (steps - 1)
    s.close()


def test_noalloc_refuses_unmatched_duplicate_and_bad_tensors(env):
    """A row that lists a neighbour twice while the neighbour lists it once is
    asymmetric as a multiset and is refused by the validation kernel before
    any schedule is built; tensors of the wrong type or size are refused by
    the binding before a pointer is passed."""
    pg, torch = env
    inst = W.gnm(200, 500, seed=3)
    rp, col, wt = inst.row_ptr.astype(np.int64), inst.col.astype(np.int32), inst.w.astype(np.int32)
    i = int(np.argmax(np.diff(rp) > 0))
    e = int(rp[i])
    col2 = np.insert(col, e, col[e])                 # row i lists col[e] twice
    w2 = np.insert(wt, e, wt[e])
    rp2 = rp.copy()
    rp2[i + 1:] += 1
    d_rp = torch.from_numpy(rp2.astype(np.int32)).cuda()
    d_col = torch.from_numpy(col2).cuda()
    d_w = torch.from_numpy(w2).cuda()
    R, n = 4, inst.n
    x = torch.ones((R, n), dtype=torch.int8, device="cuda")
    E = torch.empty(R, dtype=torch.int64, device="cuda")
    with pytest.raises(pg.PamcError) as ei:
        pg.pamc_sweeps_noalloc(n, int(rp2[-1]), d_rp, d_col, d_w, 127, 0, R, 1, 0.5, 1, 0, x, x, E)
    assert ei.value.status == 2
    # the scratch still serves a valid instance afterwards
    rp_ok, col_ok, w_ok, H = _dev_csr(torch, inst)
    pg.pamc_sweeps_noalloc(n, inst.nnz, rp_ok, col_ok, w_ok, H, 0, R, 1, 0.5, 1, 0, x, x, E)
    for bad in (dict(E=torch.empty(R, dtype=torch.int32, device="cuda")),
                dict(x=torch.ones((R, n - 1), dtype=torch.int8, device="cuda")),
                dict(x=torch.ones((R, n), dtype=torch.int8))):
        a = dict(x=x, E=E)
        a.update(bad)
        with pytest.raises(ValueError):
            pg.pamc_sweeps_noalloc(n, inst.nnz, rp_ok, col_ok, w_ok, H, 0, R, 1, 0.5, 1, 0, a["x"], a["x"],
                                   a["E"])
