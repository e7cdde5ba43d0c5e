"""Batched execution: every member of a batch computes exactly what it computes
alone (spins, energies, parents, copy counts, controller state and best cut),
whatever joins or leaves the batch meanwhile, and one member is checked against
the oracle directly.  The serving loop returns the same cut and configuration
for each request as the one-instance-at-a-time path."""
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


def _max_degree_graph(n, m, dmax, seed, **kw):
    from test_gpu_parity import _max_degree_graph as g
    return g(n, m, dmax, seed, **kw)


def mix():
    """Instances of every size class (n <= 2048, <= 8192, larger), both weight
    kinds, CSR and ELL sweeps, ragged R, both update rules."""
    return [
        (W.erdos_renyi(300, 0.05, signed=False, seed=1), dict(R=64, sweeps=2, steps=21, rule=0, seed=11)),
        (W.gnm(1500, 4300, signed=True, seed=2), dict(R=50, sweeps=3, steps=34, rule=1, seed=12)),
        (W.torus(60, 60, signed=True, seed=3), dict(R=96, sweeps=2, steps=19, rule=0, seed=13)),
        (W.torus(30, 30, signed=False, seed=6), dict(R=20, sweeps=0, steps=9, rule=0, seed=16)),
        (W.er_avg_degree(9000, 12, signed=True, seed=4), dict(R=36, sweeps=1, steps=18, rule=0, seed=14)),
        (W.er_avg_degree(2100, 20, signed=False, seed=5), dict(R=128, sweeps=2, steps=40, rule=1, seed=15,
                                                            z_rst=13, restart_reinit=0)),
        # field ranges that fit 4-bit lanes: eight replicas a word in the
        # batch as alone -- the fixed bias (ELL widths 4 and 8) and the biased
        # lanes (half-row ranges <= 15 on widths 12 and 16, weighted too; the
        # signed gnm member above as well), ragged groups of eight, both rules
        (W.torus(80, 80, signed=True, seed=8), dict(R=28, sweeps=2, steps=15, rule=1, seed=17)),
        (_max_degree_graph(1200, 3500, 7, 9), dict(R=20, sweeps=2, steps=12, rule=0, seed=18)),
        (_max_degree_graph(2500, 13000, 16, 10, weights=(-2, -1, 1, 1)), dict(R=44, sweeps=2, steps=14, rule=1,
                                                                           seed=19)),
        (_max_degree_graph(900, 4000, 12, 11), dict(R=12, sweeps=1, steps=10, rule=0, seed=20)),
    ]


def snapshot(pg, h, n, R):
    spins, E, par, cnt = pg.pamc_state(h, R, n)
    m, b = pg.pamc_best(h, n)
    return dict(spins=spins, E=E, par=par, cnt=cnt, best=(m, b), ctl=pg.pamc_control_state(h))


def assert_same(a, b, where):
    for k in ("spins", "E", "par", "cnt"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=f"{k} {where}")
    assert a["best"][0] == b["best"][0], f"M* {where}"
    np.testing.assert_array_equal(a["best"][1], b["best"][1], err_msg=f"best spins {where}")
    for k, v in a["ctl"].items():
        assert v == b["ctl"][k], f"ctl {k} {where}: {v} != {b['ctl'][k]}"


def alone(pg, inst, p):
    h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
    pg.pamc_run(h, **p)
    s = snapshot(pg, h, inst.n, p["R"])
    pg.pamc_destroy(h)
    return s


@pytest.mark.parametrize("push", ["0", "1"])
def test_batch_members_equal_alone(pg, monkeypatch, push):
    """Also with the push-model sweep for the members it applies to (field
    range <= 63, ELL schedules, one lane per vertex), in and out of the batch."""
    monkeypatch.setenv("PAMC_SWEEP_PUSH", push)
    cases = mix()
    ref = [alone(pg, inst, p) for inst, p in cases]
    b = pg.pamc_batch_create(0)
    hs = []
    try:
        # staggered joins: two members first, the rest after some steps
        for i, (inst, p) in enumerate(cases):
            h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
            pg.pamc_init(h, **p)
            hs.append(h)
        pg.pamc_batch_add(b, hs[0])
        pg.pamc_batch_add(b, hs[1])
        pg.pamc_batch_step(b, 5)
        for h in hs[2:]:
            pg.pamc_batch_add(b, h)
        got = {}
        while pg.pamc_batch_size(b) > 0:
            pg.pamc_batch_step(b, 3)
            for h in pg.pamc_batch_retire(b):
                i = [x.value for x in hs].index(h.value)
                inst, p = cases[i]
                got[i] = snapshot(pg, h, inst.n, p["R"])
        assert sorted(got) == list(range(len(cases)))
        for i in range(len(cases)):
            assert_same(got[i], ref[i], f"member {i} ({cases[i][0].name})")
        assert pg.pamc_batch_graph_builds(b) >= 2
    finally:
        for h in hs:
            pg.pamc_destroy(h)
        pg.pamc_batch_destroy(b)


def test_batch_member_matches_oracle(pg):
    inst = W.erdos_renyi(200, 0.06, signed=True, seed=7)
    p = dict(R=40, sweeps=2, steps=20, rule=0, seed=5, beta0=0.2, beta1=2.5)
    ref = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **p)
    ref.step(p["steps"])
    other = W.torus(20, 20, signed=True, seed=8)
    b = pg.pamc_batch_create(0)
    h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
    h2 = pg.pamc_create_csr(other.n, other.row_ptr, other.col, other.w)
    try:
        pg.pamc_init(h, **p)
        pg.pamc_init(h2, R=64, sweeps=3, steps=50, seed=9)
        pg.pamc_batch_add(b, h2)
        pg.pamc_batch_add(b, h)
        pg.pamc_batch_step(b, p["steps"])
        pg.pamc_batch_sync(b)
        spins, E, par, cnt = pg.pamc_state(h, p["R"], inst.n)
        np.testing.assert_array_equal(spins, ref.spins())
        np.testing.assert_array_equal(E, ref.energy())
        rp, rc = ref.parents()
        np.testing.assert_array_equal(par, rp)
        np.testing.assert_array_equal(cnt, rc)
        m, bs = pg.pamc_best(h, inst.n)
        rm, rb = ref.best()
        assert m == rm
        np.testing.assert_array_equal(bs, rb)
    finally:
        pg.pamc_destroy(h)
        pg.pamc_destroy(h2)
        pg.pamc_batch_destroy(b)


def test_join_after_stepping_alone(pg):
    """A handle stepped on its own for a while (schedule ring partly used) and
    then moved into a batch ends exactly where a run alone ends."""
    inst = W.gnm(900, 2600, signed=True, seed=21)
    p = dict(R=72, sweeps=2, steps=45, rule=0, seed=3)
    ref = alone(pg, inst, p)
    for pre in (5, 16, 17):
        h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
        b = pg.pamc_batch_create(0)
        try:
            pg.pamc_init(h, **p)
            pg.pamc_step(h, pre)
            pg.pamc_sync(h)
            pg.pamc_batch_add(b, h)
            pg.pamc_batch_step(b, p["steps"])
            assert len(pg.pamc_batch_retire(b)) == 1
            assert_same(snapshot(pg, h, inst.n, p["R"]), ref, f"joined after {pre} steps")
        finally:
            pg.pamc_destroy(h)
            pg.pamc_batch_destroy(b)


def test_finished_member_is_frozen_and_target_stop(pg):
    """A member past its last step does nothing while the others go on; a
    member that reaches its target cut stops as it does alone."""
    a = W.torus(16, 16, signed=True, seed=31)
    c = W.erdos_renyi(150, 0.08, signed=False, seed=32)
    pa = dict(R=32, sweeps=2, steps=6, seed=1)
    pc = dict(R=32, sweeps=2, steps=30, seed=2)
    ra = alone(pg, a, pa)
    # target: the cut the run alone reaches after 10 steps
    h = pg.pamc_create_csr(c.n, c.row_ptr, c.col, c.w)
    pg.pamc_init(h, **pc)
    pg.pamc_step(h, 10)
    target, _ = pg.pamc_best(h, c.n)
    pg.pamc_destroy(h)
    pc["target_cut"] = int(target)
    rc = alone(pg, c, pc)
    assert rc["ctl"]["done"] == 1
    b = pg.pamc_batch_create(0)
    ha = pg.pamc_create_csr(a.n, a.row_ptr, a.col, a.w)
    hc = pg.pamc_create_csr(c.n, c.row_ptr, c.col, c.w)
    try:
        pg.pamc_init(ha, **pa)
        pg.pamc_init(hc, **pc)
        pg.pamc_batch_add(b, ha)
        pg.pamc_batch_add(b, hc)
        pg.pamc_batch_step(b, 40)   # a finishes after 6 steps and stays in the graph
        pg.pamc_batch_sync(b)
        assert pg.pamc_batch_active(b) == 0
        assert_same(snapshot(pg, ha, a.n, pa["R"]), ra, "finished member")
        assert_same(snapshot(pg, hc, c.n, pc["R"]), rc, "member stopped at its target")
        assert len(pg.pamc_batch_retire(b)) == 2
    finally:
        pg.pamc_destroy(ha)
        pg.pamc_destroy(hc)
        pg.pamc_batch_destroy(b)


def test_batch_device_memory_placement(pg):
    """Size classes whose Ising groups keep their spin words in device memory
    give every member what it computes alone (placement changes speed only),
    next to classes on chip and Potts members."""
    cases = mix()[:5] + [(W.gnm(700, 4200, signed=False, seed=21), dict(kind=1, R=24, sweeps=2, steps=15,
                                                                       seed=31))]
    ref = [alone(pg, inst, p) for inst, p in cases]
    b = pg.pamc_batch_create(0)
    hs = []
    try:
        pg.pamc_batch_set_placement(b, 0, True)
        pg.pamc_batch_set_placement(b, 2, True)
        assert pg.pamc_batch_get_placement(b, 0) and not pg.pamc_batch_get_placement(b, 1)
        for inst, p in cases:
            h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
            pg.pamc_init(h, **p)
            pg.pamc_batch_add(b, h)
            hs.append(h)
        pg.pamc_batch_step(b, 3)
        pg.pamc_batch_set_placement(b, 1, True)          # a change between steps takes effect at the next
        while pg.pamc_batch_active(b) > 0:
            pg.pamc_batch_step(b, 4)
        pg.pamc_batch_sync(b)
        for (inst, p), h, r in zip(cases, hs, ref):
            assert_same(snapshot(pg, h, inst.n, p["R"]), r, inst.name)
    finally:
        pg.pamc_batch_destroy(b)
        for h in hs:
            pg.pamc_destroy(h)


def test_batch_max_cut_and_max3cut_members(pg):
    """Max-3-Cut members (three-state Potts, cascaded sampler) share batches
    with Max-Cut members: every member of every size class, ELL or CSR
    schedules, ragged R, equals its run alone after every few steps, and a
    Potts member equals the oracle."""
    cases = [
        (W.gnm(700, 4200, signed=False, seed=21), dict(kind=1, R=24, sweeps=2, steps=15, seed=31)),
        (W.torus(40, 40, signed=True, seed=22), dict(kind=0, R=32, sweeps=2, steps=12, seed=32)),
        (W.er_avg_degree(3000, 12, signed=True, seed=23), dict(kind=1, R=18, sweeps=1, steps=14, seed=33,
                                                               z_rst=6, restart_reinit=0)),
        (W.er_avg_degree(9500, 8, signed=False, seed=24), dict(kind=1, R=12, sweeps=2, steps=9, seed=34)),
        (W.gnm(400, 700, signed=True, seed=25), dict(kind=0, R=20, sweeps=3, steps=16, rule=1, seed=35)),
    ]
    ref = [alone(pg, inst, p) for inst, p in cases]
    inst0, p0 = cases[0]
    orc = oracle.OracleRun(inst0.row_ptr, inst0.col, inst0.w, **p0)
    orc.step(p0["steps"])
    b = pg.pamc_batch_create(0)
    hs = []
    try:
        for inst, p in cases:
            h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
            pg.pamc_init(h, **p)
            pg.pamc_batch_add(b, h)
            hs.append(h)
        while pg.pamc_batch_active(b) > 0:
            pg.pamc_batch_step(b, 4)
        pg.pamc_batch_sync(b)
        for (inst, p), h, r in zip(cases, hs, ref):
            assert_same(snapshot(pg, h, inst.n, p["R"]), r, inst.name)
        spins, E, _, _ = pg.pamc_state(hs[0], p0["R"], inst0.n)
        np.testing.assert_array_equal(spins, orc.spins())
        np.testing.assert_array_equal(E, orc.energy())
        assert pg.pamc_best(hs[0], inst0.n)[0] == orc.best()[0]
    finally:
        pg.pamc_batch_destroy(b)
        for h in hs:
            pg.pamc_destroy(h)


def test_batch_augmented_members_equal_alone(pg):
    """Members with the stagnation controller (reheats and cluster moves,
    run per member in the batch) and with restarts that re-draw the
    population (in the batch, after the controller) end exactly as they do
    alone -- Max-Cut on byte and 4-bit lanes, both rules, and Max-3-Cut --
    joining at different steps, beside plain members."""
    aug = dict(stagnation=1, win_short=2, win_long=3, cooldown_tau=1)
    cases = [
        (W.torus(40, 40, signed=True, seed=31), dict(R=64, sweeps=2, steps=40, rule=0, z_rst=17, seed=41, **aug)),
        (W.gnm(1500, 4300, signed=True, seed=32), dict(R=44, sweeps=2, steps=36, rule=1, z_rst=13, seed=42, **aug)),
        (W.gnm(900, 3600, signed=False, seed=33), dict(kind=1, R=24, sweeps=2, steps=30, z_rst=11, seed=43)),
        (W.er_avg_degree(9000, 12, signed=True, seed=34), dict(R=20, sweeps=1, steps=25, z_rst=8, seed=44, **aug)),
        (W.erdos_renyi(300, 0.05, signed=False, seed=35), dict(R=32, sweeps=2, steps=20, seed=45)),
    ]
    ref = [alone(pg, inst, p) for inst, p in cases]
    b = pg.pamc_batch_create(0)
    hs = []
    try:
        for inst, p in cases:
            h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
            pg.pamc_init(h, **p)
            hs.append(h)
        pg.pamc_step(hs[1], 14)      # steps alone past its first restart, then joins
        pg.pamc_batch_add(b, hs[0])
        pg.pamc_batch_add(b, hs[1])
        pg.pamc_batch_add(b, hs[2])
        pg.pamc_batch_step(b, 6)
        for h in hs[3:]:
            pg.pamc_batch_add(b, h)
        got = {}
        while pg.pamc_batch_size(b) > 0:
            pg.pamc_batch_step(b, 4)
            for h in pg.pamc_batch_retire(b):
                i = [x.value for x in hs].index(h.value)
                inst, p = cases[i]
                got[i] = snapshot(pg, h, inst.n, p["R"])
        assert sorted(got) == list(range(len(cases)))
        for i in range(len(cases)):
            assert_same(got[i], ref[i], f"member {i} ({cases[i][0].name})")
            if cases[i][1].get("stagnation"):
                assert got[i]["ctl"]["ncm_flipped"] > 0, i
            if cases[i][1].get("z_rst"):
                assert got[i]["ctl"]["cycle"] >= 1, i
    finally:
        for h in hs:
            pg.pamc_destroy(h)
        pg.pamc_batch_destroy(b)


def test_batch_refusals(pg):
    inst = W.torus(8, 8, signed=True, seed=1)
    b = pg.pamc_batch_create(0)
    h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
    try:
        with pytest.raises(pg.PamcError):
            pg.pamc_batch_add(b, h)                       # not initialised
        pg.pamc_init(h, R=16, steps=5, kind=1, rule=2, K=4)
        with pytest.raises(pg.PamcError):
            pg.pamc_batch_add(b, h)                       # softmax Potts members are refused
        pg.pamc_init(h, R=16, steps=5)
        pg.pamc_batch_add(b, h)
        with pytest.raises(pg.PamcError):
            pg.pamc_batch_add(b, h)                       # already a member
        assert pg.pamc_footprint(h, R=16, steps=5) > 16 * inst.n * 2
    finally:
        pg.pamc_batch_destroy(b)
        pg.pamc_destroy(h)


def test_server_equals_sequential(pg):
    from paper_2606_25203_gb300.serving import Server, serve_sequential
    reqs = W.serving_stream(12, rate=400.0, seed=3, n_lo=300, n_hi=5000, er_degree=10.0, max3cut_frac=0.4)
    assert 0 < sum(r.kind for r in reqs) < len(reqs)      # Max-Cut and Max-3-Cut requests
    params = dict(R=64, sweeps=2, steps=24, beta0=0.1, beta1=3.0, seed=17)
    seq = serve_sequential(reqs, params, keep_spins=True)
    # a small budget forces admission to wait for retirements
    srv = Server(hbm_budget=40 << 20, max_active=4, steps_per_tick=3, keep_spins=True)
    try:
        st = srv.serve(reqs, params)
    finally:
        srv.close()
    assert len(st.results) == len(reqs)
    assert st.peak_active <= 4
    a = {r.rid: r for r in seq.results}
    for r in st.results:
        assert r.cut == a[r.rid].cut, f"request {r.rid}"
        np.testing.assert_array_equal(r.spins, a[r.rid].spins, err_msg=f"request {r.rid}")
        assert r.finished >= r.admitted >= r.arrival - 1e-9


def test_served_stream_requests_match_oracle(pg):
    """Requests drawn by the configuration-5 generator at its own settings (N
    in [800, 20000], Erdos-Renyi unit and +-1 weights of degree 20 and +-1
    tori, a quarter Max-3-Cut): the six smallest of forty, served through the
    batching server with a small budget, each end with the oracle's best cut
    and configuration (fewer replicas and steps than the stream's, so that
    the oracle finishes in seconds)."""
    from paper_2606_25203_gb300.serving import Server
    stream = W.serving_stream(40, rate=400.0, seed=11, max3cut_frac=0.25)
    reqs = sorted(stream, key=lambda r: r.inst.n)[:6]
    assert {r.kind for r in reqs} == {0, 1}, [(r.inst.name, r.kind) for r in reqs]
    params = dict(R=32, sweeps=2, steps=12, beta0=0.1, beta1=3.0, seed=23)
    srv = Server(hbm_budget=64 << 20, max_active=3, steps_per_tick=4, keep_spins=True)
    try:
        st = srv.serve(reqs, params)
    finally:
        srv.close()
    got = {r.rid: r for r in st.results}
    assert len(got) == len(reqs)
    for req in reqs:
        ref = oracle.OracleRun(req.inst.row_ptr, req.inst.col, req.inst.w, kind=req.kind, **params)
        ref.step(params["steps"])
        cut, spins = ref.best()
        assert got[req.rid].cut == cut, f"request {req.rid} ({req.inst.name}, kind {req.kind})"
        np.testing.assert_array_equal(got[req.rid].spins, spins, err_msg=f"request {req.rid}")


def test_shapes_change_speed_not_results(pg):
    """Every launch shape of every size class gives the same members' results,
    and the autotuner sets one of the candidates."""
    from paper_2606_25203_gb300.tune import tune_batch_shapes
    cases = [(W.gnm(1200, 3400, signed=True, seed=41), dict(R=40, sweeps=2, steps=7, seed=1)),
             (W.er_avg_degree(3000, 16, signed=False, seed=42), dict(R=24, sweeps=2, steps=7, seed=2, rule=1)),
             (W.torus(95, 95, signed=True, seed=43), dict(R=28, sweeps=1, steps=7, seed=3))]
    ref = [alone(pg, inst, p) for inst, p in cases]
    for shape, lanes in [((1, 1), 1), ((2, 16), 1), ((8, 4), 1), ((3, 3), 1), ((1, 8), 2), ((2, 16), 4),
                         ((1, 32), 4)]:
        b = pg.pamc_batch_create(0)
        hs = []
        try:
            for c in range(3):
                pg.pamc_batch_set_shape(b, c, *shape)
                pg.pamc_batch_set_lanes(b, c, lanes)
                assert pg.pamc_batch_get_shape(b, c) == shape
                assert pg.pamc_batch_get_lanes(b, c) == lanes
            for inst, p in cases:
                h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
                pg.pamc_init(h, **p)
                pg.pamc_batch_add(b, h)
                hs.append(h)
            pg.pamc_batch_step(b, 7)
            pg.pamc_batch_sync(b)
            for i, (inst, p) in enumerate(cases):
                assert_same(snapshot(pg, hs[i], inst.n, p["R"]), ref[i], f"shape {shape} lanes {lanes} member {i}")
        finally:
            pg.pamc_batch_destroy(b)
            for h in hs:
                pg.pamc_destroy(h)
    b = pg.pamc_batch_create(0)
    try:
        with pytest.raises(pg.PamcError):
            pg.pamc_batch_set_shape(b, 0, 8, 8)      # 64 warps
        with pytest.raises(pg.PamcError):
            pg.pamc_batch_set_shape(b, 3, 1, 1)      # no such class
        with pytest.raises(pg.PamcError):
            pg.pamc_batch_set_lanes(b, 0, 3)         # 1, 2 or 4
        got = tune_batch_shapes(b, [c[0] for c in cases], dict(R=32, sweeps=1), steps=1, rounds=1,
                                candidates=((1, 4), (2, 2), (1, 8, 2), (1, 8, 1, 1)))
        assert sorted(got) == [0, 1, 2]
        for c, (g, w, lv, ms, gm) in got.items():
            assert (g, w, lv, gm) in ((1, 4, 1, 0), (2, 2, 1, 0), (1, 8, 2, 0), (1, 8, 1, 1)) and ms > 0
            assert pg.pamc_batch_get_shape(b, c) == (g, w)
            assert pg.pamc_batch_get_lanes(b, c) == lv
            assert pg.pamc_batch_get_placement(b, c) == bool(gm)
    finally:
        pg.pamc_batch_destroy(b)
