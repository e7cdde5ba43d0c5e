"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every comparison is exact: spins, energies, parents, copy counts, the best cut
and configuration, and the controller state (t, z, cycle, cooldown, flags,
beta and Delta bit for bit) after every iteration.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

CTL_EXACT = ("t", "z", "cycle", "cooldown", "enable_cm", "done", "ncm_last", "hist_len",
             "ncm_flipped", "ncm_dE_max")


@pytest.fixture(scope="module")
def pg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_25203_gb300 as pg
    pg.load()
    return pg


def compare_run(pg, inst, steps, check_every=1, **params):
    ref = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, steps=steps, **params)
    s = pg.Solver(inst.row_ptr, inst.col, inst.w)
    s.init(steps=steps, **params)
    assert pg.pamc_weight_sum(s.h) == ref.weight_sum()
    done = 0
    while done < steps:
        k = min(check_every, steps - done)
        s.step(k)
        ref.step(k)
        done += k
        spins, E, par, cnt = s.state()
        where = f"after {done} steps"
        np.testing.assert_array_equal(spins, ref.spins(), err_msg=f"spins {where}")
        np.testing.assert_array_equal(E, ref.energy(), err_msg=f"energies {where}")
        rp, rc = ref.parents()
        np.testing.assert_array_equal(par, rp, err_msg=f"parents {where}")
        np.testing.assert_array_equal(cnt, rc, err_msg=f"counts {where}")
        gc, oc = s.control(), ref.ctl()
        for key in CTL_EXACT:
            assert gc[key] == oc[key], f"{key} {where}: {gc[key]} != {oc[key]}"
        assert gc["beta"] == oc["beta"] and gc["delta"] == oc["delta"], where
        m, b = s.best()
        rm, rb = ref.best()
        assert m == rm, f"M* {where}"
        np.testing.assert_array_equal(b, rb, err_msg=f"best spins {where}")
    launches = s.launches()
    s.close()
    return ref, launches


@pytest.mark.parametrize("rule", [0, 1])
def test_conventional_pamc_er(pg, rule):
    inst = W.erdos_renyi(150, 0.08, signed=False, seed=3)
    compare_run(pg, inst, 12, R=20, sweeps=3, beta0=0.1, beta1=3.0, rule=rule, seed=7)


def test_signed_sparse_ragged_population(pg):
    # R not a multiple of the replica group, n not a multiple of 16
    inst = W.gnm(333, 900, signed=True, seed=2)
    compare_run(pg, inst, 10, R=13, sweeps=2, beta0=0.2, beta1=2.5, seed=11)


def test_potts_max3cut(pg):
    inst = W.gnm(300, 1800, signed=False, seed=4)
    compare_run(pg, inst, 12, kind=1, R=10, sweeps=2, beta0=0.1, beta1=3.0, seed=5)


def test_potts_signed(pg):
    inst = W.erdos_renyi(120, 0.1, signed=True, seed=9)
    compare_run(pg, inst, 8, kind=1, R=7, sweeps=3, beta0=0.3, beta1=2.0, seed=2)


@pytest.mark.parametrize("K,gamma", [(3, 1.0), (2, 0.5), (4, 0.0), (5, 2.5), (8, 1.0)])
def test_potts_softmax_noisy_argmax(pg, K, gamma):
    # Sec. III.F softmax update, K labels, ragged R
    inst = W.gnm(260, 1300, signed=K % 2 == 0, seed=K)
    compare_run(pg, inst, 9, kind=1, rule=2, K=K, gamma=gamma, R=22, sweeps=2, beta0=0.1, beta1=3.0,
                seed=3 + K)


def test_potts_softmax_torus_restart_and_sa(pg):
    inst = W.torus(18, 18, signed=True, seed=5)
    compare_run(pg, inst, 30, kind=1, rule=2, K=3, gamma=0.7, R=40, sweeps=2, beta0=0.2, beta1=4.0,
                z_rst=13, seed=9)
    compare_run(pg, inst, 5, kind=1, rule=2, K=6, gamma=1.2, R=9, sweeps=3, resample=0, seed=2)


def test_potts_rejects_bad_k(pg):
    inst = W.torus(6, 6, signed=True, seed=1)
    h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
    try:
        for bad in (dict(kind=1, rule=0, K=4), dict(kind=1, rule=2, K=9), dict(kind=1, rule=2, K=1),
                    dict(kind=1, rule=2, K=3, gamma=-1.0), dict(kind=1, rule=1)):
            with pytest.raises(pg.PamcError):
                pg.pamc_init(h, R=8, steps=2, **bad)
    finally:
        pg.pamc_destroy(h)


def test_augmented_pamc_with_ncm_and_restart(pg):
    inst = W.torus(16, 16, signed=True, seed=2)
    ref, _ = compare_run(pg, inst, 150, R=32, sweeps=2, beta0=0.5, beta1=6.0, stagnation=1,
                         z_rst=120, cooldown_tau=5, seed=3)
    st = ref.ctl()
    assert st["ncm_flipped"] > 0 and st["cycle"] == 1


@pytest.mark.parametrize("R,n_top", [(24, 7), (40, 11)])
def test_augmented_ncm_ragged_population(pg, R, n_top):
    """Cluster moves on populations that are not a power of two, with more
    targets than the default: the (energy, slot) sort that picks the targets
    pads to the next power of two, and the targets' moves, the energies and
    the controller stay bit for bit the oracle's."""
    inst = W.torus(16, 16, signed=True, seed=2)
    ref, _ = compare_run(pg, inst, 150, R=R, sweeps=2, beta0=0.5, beta1=6.0, stagnation=1,
                         z_rst=120, cooldown_tau=5, n_top=n_top, seed=3)
    assert ref.ctl()["ncm_flipped"] > 0


def test_augmented_potts_controller(pg):
    inst = W.gnm(200, 1000, signed=False, seed=8)
    compare_run(pg, inst, 90, kind=1, R=16, sweeps=1, beta0=0.5, beta1=5.0, stagnation=1,
                z_rst=70, cooldown_tau=4, seed=4)


@pytest.mark.parametrize("cfg,rule", [("1,1,2", 0), ("1,1,4", 1), ("1,1,8", 0), ("2,2,8", 1), ("3,4,4", 0),
                                      ("1,2,16", 1), ("2,4,32", 0), ("1,32,32", 1)])
def test_lanes_per_vertex_shapes(pg, monkeypatch, cfg, rule):
    """Several lanes per vertex (coupling slots split, partial sums shuffled)
    give the sequential result: dense ER rows longer than the lanes' share,
    sparse rows shorter than it, a ragged population, both update rules."""
    monkeypatch.setenv("PAMC_SWEEP_CFG", cfg)
    monkeypatch.setenv("PAMC_SWEEP_NIBBLE", "0")    # the gnm rows would take the 4-bit lanes (one lane a vertex)
    lpv = int(cfg.split(",")[2])
    for inst, R in ((W.erdos_renyi(300, 0.2, signed=True, seed=4), 13),
                    (W.gnm(333, 900, signed=True, seed=2), 20)):
        s = pg.Solver(inst.row_ptr, inst.col, inst.w)
        s.init(R=R, sweeps=2, steps=3, rule=rule, seed=9)
        assert pg.pamc_sweep_shape(s.h)[2] == lpv
        s.close()
        compare_run(pg, inst, 6, R=R, sweeps=2, beta0=0.3, beta1=3.0, rule=rule, stagnation=1,
                    z_rst=4, cooldown_tau=1, seed=9)


@pytest.mark.parametrize("rule", [0, 2])
def test_potts_launch_shapes_same_results(pg, monkeypatch, rule):
    """Potts sweeps under several forced launch shapes (groups per CTA,
    warps per group; lane pairs for the cascaded sampler and quads of lanes
    for the softmax one -- several lanes a position, rows longer than 16
    slots, levels that leave pairs or quads idle, a ragged population) give
    the oracle's labels and energies."""
    inst = W.gnm(700, 4200, signed=False, seed=12)
    assert int(np.diff(inst.row_ptr).max()) > 16
    params = dict(kind=1, rule=rule, R=26, sweeps=2, beta0=0.2, beta1=2.5, seed=6)
    if rule == 2:
        params.update(K=3, gamma=1.0)
    for cfg in ("1,1", "1,4", "3,2", "2,8", "1,1,2", "1,8,2", "3,2,2", "1,1,4", "1,8,4", "2,4,4"):
        monkeypatch.setenv("PAMC_SWEEP_CFG", cfg)
        lanes = int(cfg.split(",")[2]) if cfg.count(",") == 2 else 1
        want = lanes if (rule, lanes) in ((0, 2), (2, 4)) else 1
        s = pg.Solver(inst.row_ptr, inst.col, inst.w)
        s.init(steps=4, **params)
        assert pg.pamc_sweep_shape(s.h)[2] == want, cfg
        s.close()
        compare_run(pg, inst, 4, **params)


def test_lanes_per_vertex_default_choice(pg, monkeypatch):
    """Narrow-level dense-row instances get several lanes per vertex; the
    torus (rows of four) keeps one."""
    monkeypatch.delenv("PAMC_SWEEP_CFG", raising=False)
    for inst, want_many in ((W.c1_er800(), True), (W.torus(40, 40, signed=True, seed=1), False)):
        s = pg.Solver(inst.row_ptr, inst.col, inst.w)
        s.init(R=128, sweeps=2, steps=3, seed=0)
        lpv = pg.pamc_sweep_shape(s.h)[2]
        s.close()
        assert (lpv > 1) == want_many, (inst.name, lpv)


def test_independent_chains_baseline(pg):
    inst = W.gnm(400, 1100, signed=True, seed=6)
    compare_run(pg, inst, 6, R=9, sweeps=2, resample=0, seed=1)


def test_target_cut_terminates(pg):
    inst = W.erdos_renyi(16, 0.4, signed=False, seed=0)
    ref = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, R=64, sweeps=2, steps=40, beta0=0.1,
                           beta1=3.0)
    ref.step(40)
    target = ref.best()[0]
    _, _ = compare_run(pg, inst, 60, R=64, sweeps=2, beta0=0.1, beta1=3.0, target_cut=target)


def test_degenerate_sizes(pg):
    # a single vertex with no edges, and a single replica
    one = W.csr_from_edges(1, np.zeros(0), np.zeros(0), np.zeros(0), "one")
    compare_run(pg, one, 3, R=3, sweeps=2)
    inst = W.gnm(50, 80, signed=True, seed=3)
    compare_run(pg, inst, 5, R=1, sweeps=1)
    # zero sweeps: resampling and control only
    compare_run(pg, inst, 5, R=8, sweeps=0)


def test_config_er800_full(pg):
    """ER N=800 p=0.06 unit weights, R=128, 50 steps x 5 sweeps, beta 0.1->3.0."""
    inst = W.c1_er800()
    compare_run(pg, inst, 50, check_every=5, R=128, sweeps=5, beta0=0.1, beta1=3.0, seed=0)


def test_torus141_multi_level_tiles(pg):
    """Torus 141x141 at reduced R and steps: many levels, many warps per group."""
    inst = W.c2a_torus141()
    compare_run(pg, inst, 3, R=12, sweeps=3, beta0=0.1, beta1=4.0, seed=0)


def test_sparse7000_augmented_reduced(pg):
    inst = W.c2b_sparse7000()
    compare_run(pg, inst, 4, R=16, sweeps=4, beta0=0.1, beta1=4.0, stagnation=1, z_rst=400,
                seed=0)


def test_potts2000_reduced(pg):
    inst = W.c3_sparse2000()
    compare_run(pg, inst, 5, kind=1, R=12, sweeps=4, beta0=0.1, beta1=3.0, seed=0)


@pytest.mark.parametrize("name", ["torus", "sparse7000"])
def test_full_size_population_sampled(pg, name):
    """R=4096 at the benchmark's launch configuration.  Replicas are
    independent until the first resampling, so the oracle can reproduce a
    sample of them one by one; the rest is checked by properties that hold
    at any size (population conserved, energies equal the definition)."""
    inst = W.c2a_torus141() if name == "torus" else W.c2b_sparse7000()
    R = 4096
    s = pg.Solver(inst.row_ptr, inst.col, inst.w)
    s.init(R=R, sweeps=10, steps=500, beta0=0.1, beta1=4.0, stagnation=1, z_rst=400, seed=0)
    s.step(1)
    spins, E, par, cnt = s.state()
    ref = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, R=8, sweeps=10, steps=500, beta0=0.1,
                           beta1=4.0, stagnation=1, z_rst=400, seed=0)
    ref.step(1)
    np.testing.assert_array_equal(spins[:8], ref.spins())
    np.testing.assert_array_equal(E[:8], ref.energy())
    s.step(2)
    spins, E, par, cnt = s.state()
    assert cnt.sum() == R and np.all(np.diff(par) >= 0)
    rng = np.random.default_rng(0)
    for r in rng.choice(R, size=16, replace=False):
        assert E[r] == oracle.energy_ising(inst.row_ptr, inst.col, -inst.w, spins[r])
    m, b = s.best()
    assert m == (pg.pamc_weight_sum(s.h) - oracle.energy_ising(inst.row_ptr, inst.col, -inst.w, b)) // 2
    s.close()


@pytest.mark.parametrize("rule", [0, 2])
def test_potts_full_size_first_step(pg, rule):
    """Configuration 3 at full size: N=2,000 (avg degree 12), R=2,048, 10
    sweeps, the benchmark's launch shape.  The first iteration does not
    resample, so the oracle runs all 2,048 replicas through it and every label
    and energy is compared; the cascaded sampler and the softmax noisy argmax."""
    inst = W.c3_sparse2000()
    params = dict(kind=1, rule=rule, R=2048, sweeps=10, steps=300, beta0=0.1, beta1=3.0, seed=0)
    if rule == 2:
        params.update(K=3, gamma=1.0)
    s = pg.Solver(inst.row_ptr, inst.col, inst.w)
    s.init(**params)
    s.step(1)
    spins, E, _, _ = s.state()
    ref = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **params)
    ref.step(1)
    np.testing.assert_array_equal(spins, ref.spins())
    np.testing.assert_array_equal(E, ref.energy())
    s.close()


def _hub_instance(n=300, seed=3):
    """Vertex 0 coupled to 63 others with +-1 weights (sum |w| = 63, the
    largest field range of the push-model sweep), weights +-1 and +-2 on a
    random rest of average degree 19."""
    rng = np.random.default_rng(seed)
    ei, ej, w = [], [], []
    for j in range(1, 64):
        ei.append(0); ej.append(j); w.append(int(rng.choice([-1, 1])))
    pairs = set()
    while len(pairs) < 2200:     # dense enough that the schedules use the ELL rows
        a, b = (int(x) for x in rng.integers(64, n, size=2))
        if a != b:
            pairs.add((min(a, b), max(a, b)))
    for a, b in sorted(pairs):
        ei.append(a); ej.append(b); w.append(int(rng.choice([-2, -1, 1, 2])))
    inst = W.csr_from_edges(n, np.array(ei), np.array(ej), np.array(w), "hub63")
    sums = [int(np.abs(inst.w[inst.row_ptr[i]:inst.row_ptr[i + 1]]).sum()) for i in range(n)]
    assert max(sums) == 63
    return inst


@pytest.mark.parametrize("push", ["1", "0"])
@pytest.mark.parametrize("rule", [0, 1])
def test_push_and_pull_sweeps(pg, monkeypatch, push, rule):
    """The push-model sweep (fields kept in shared memory and updated on
    flips: H <= 63, ELL schedules, one lane per vertex) and the pull sweep
    both give the oracle's spins, energies and controller, step after step:
    a torus, a ragged signed sparse graph, and a hub of field range 63 with
    weights up to 3, under both rules and several group shapes."""
    monkeypatch.setenv("PAMC_SWEEP_PUSH", push)
    monkeypatch.setenv("PAMC_SWEEP_NIBBLE", "0")     # the torus would take the 4-bit lanes
    cases = ((W.torus(20, 20, signed=True, seed=1), 13, "1,4,1"),
             (W.gnm(333, 900, signed=True, seed=2), 20, "3,2,1"),
             (_hub_instance(), 9, "2,1,1"))
    for inst, R, cfg in cases:
        monkeypatch.setenv("PAMC_SWEEP_CFG", cfg)
        s = pg.Solver(inst.row_ptr, inst.col, inst.w)
        s.init(R=R, sweeps=3, steps=3, rule=rule, seed=4)
        assert pg.pamc_sweep_mode(s.h) == (2 if push == "1" else 1), inst.name
        s.close()
        compare_run(pg, inst, 8, R=R, sweeps=3, beta0=0.2, beta1=3.0, rule=rule, stagnation=1, z_rst=6,
                    cooldown_tau=1, seed=4)


@pytest.mark.parametrize("case", ["push", "byte", "fixed4", "biased4", "wide16"])
def test_sweep_flip_count_and_timing(pg, monkeypatch, case):
    """pamc_sweep_stats: the flips counted by the sweep kernels equal the
    oracle's count over a run -- on every field-lane layout, with a ragged
    last replica group whose empty lanes must not count -- and with timing
    on every sweep launch of the handle is timed (one per step), with a
    positive device time."""
    monkeypatch.setenv("PAMC_SWEEP_PUSH", "1" if case == "push" else "0")
    monkeypatch.setenv("PAMC_SWEEP_NIBBLE", "0" if case == "byte" else "1")
    inst = {"fixed4": W.torus(16, 16, signed=True, seed=2), "wide16": _weighted_hub()}.get(
        case, W.gnm(500, 1400, signed=True, seed=5))
    want = {"push": 2, "byte": 1, "fixed4": 17, "biased4": 17, "wide16": 8}[case]
    params = dict(R=13, sweeps=3, steps=10, beta0=0.2, beta1=2.0, stagnation=1, z_rst=6, seed=8)
    if case == "wide16":
        params.update(beta0=0.01, beta1=0.3)
    ref = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **params)
    s = pg.Solver(inst.row_ptr, inst.col, inst.w)
    s.init(**params)
    assert pg.pamc_sweep_mode(s.h) == want, case
    pg.pamc_set_sweep_timing(s.h, True)
    s.step(4)
    st = pg.pamc_sweep_stats(s.h)
    ref.step(4)
    assert st["flips"] == ref.sweep_flips() and st["launches"] == 4 and st["ms"] > 0
    s.step(6)
    st = pg.pamc_sweep_stats(s.h)
    ref.step(6)
    assert st["flips"] == ref.sweep_flips() and st["launches"] == 6
    s.close()


@pytest.mark.parametrize("rule", [0, 1])
def test_group_spins_in_device_memory(pg, monkeypatch, rule):
    """The Ising sweep with the replica groups' spin words in device memory
    (PAMC_SWEEP_GLOBAL=1; chosen by itself when a group does not fit shared
    memory) gives the oracle's results step after step: ELL and CSR
    schedules, a ragged population, cluster moves and restarts."""
    monkeypatch.setenv("PAMC_SWEEP_GLOBAL", "1")
    cases = ((W.torus(20, 20, signed=True, seed=1), 13),
             (W.erdos_renyi(300, 0.2, signed=True, seed=4), 10),      # ELL padding too wide: CSR rows
             (W.gnm(500, 1400, signed=True, seed=2), 22))
    for inst, R in cases:
        s = pg.Solver(inst.row_ptr, inst.col, inst.w)
        s.init(R=R, sweeps=2, steps=3, rule=rule, seed=4)
        assert pg.pamc_sweep_mode(s.h) & 4, inst.name
        s.close()
        compare_run(pg, inst, 10, R=R, sweeps=2, beta0=0.2, beta1=3.0, rule=rule, stagnation=1, z_rst=7,
                    cooldown_tau=1, seed=4)


def _weighted_hub(n=600, hub_deg=300, wmax=2, m_rest=1500, wrest=100, seed=5):
    """A hub coupled to hub_deg vertices (weights up to wmax, degree above the
    255 an ELL record holds), and a random rest with weights up to wrest in
    magnitude: field ranges well above a byte lane."""
    rng = np.random.default_rng(seed)
    ei, ej, w = [], [], []
    for j in range(1, hub_deg + 1):
        ei.append(0); ej.append(j); w.append(int(rng.integers(1, wmax + 1)) * int(rng.choice([-1, 1])))
    pairs = set()
    while len(pairs) < m_rest:
        a, b = (int(x) for x in rng.integers(1, n, size=2))
        if a != b:
            pairs.add((min(a, b), max(a, b)))
    for a, b in sorted(pairs):
        ei.append(a); ej.append(b); w.append(int(rng.integers(-wrest, wrest + 1)) or 1)
    return W.csr_from_edges(n, np.array(ei), np.array(ej), np.array(w), f"hub{hub_deg}_w{wrest}")


@pytest.mark.parametrize("rule", [0, 1])
def test_wide_field_range_instances(pg, monkeypatch, rule):
    """Field ranges above 127 (Eq. 3 for any integer couplings up to |w| = 127
    each, sum |w| per vertex up to 32,767) run the 16-bit-lane sweep: a
    weighted hub of degree 300 (CSR rows), a random graph with weights up to
    100 (ELL rows), each against the oracle step after step with cluster
    moves and restarts; the same with the spin words in device memory."""
    insts = (_weighted_hub(), W.gnm(700, 2800, signed=True, seed=9))
    rng = np.random.default_rng(1)
    g2 = insts[1]
    g2 = W.Instance(g2.name + "_w100", g2.n, g2.row_ptr, g2.col, None)
    # symmetric weights in [-100, 100] \ {0}: draw per undirected edge
    rp, col = g2.row_ptr, g2.col
    wmap = {}
    w = np.zeros(col.shape[0], dtype=np.int32)
    for i in range(g2.n):
        for e in range(rp[i], rp[i + 1]):
            j = int(col[e])
            key = (min(i, j), max(i, j))
            if key not in wmap:
                wmap[key] = int(rng.integers(1, 101)) * int(rng.choice([-1, 1]))
            w[e] = wmap[key]
    g2.w = w
    for inst in (insts[0], g2):
        H = max(int(np.abs(inst.w[inst.row_ptr[i]:inst.row_ptr[i + 1]]).sum()) for i in range(inst.n))
        assert 127 < H <= 32767, (inst.name, H)
        for glob in ("0", "1"):
            monkeypatch.setenv("PAMC_SWEEP_GLOBAL", glob)
            s = pg.Solver(inst.row_ptr, inst.col, inst.w)
            s.init(R=10, sweeps=2, steps=3, rule=rule, seed=2)
            mode = pg.pamc_sweep_mode(s.h)
            assert mode & 8 and bool(mode & 4) == (glob == "1"), (inst.name, mode)
            s.close()
            compare_run(pg, inst, 9, R=10, sweeps=2, beta0=0.01, beta1=0.3, rule=rule, stagnation=1, z_rst=6,
                        cooldown_tau=1, seed=2)


def test_wide_field_range_refusals(pg):
    """Max-3-Cut keeps the byte-lane bound; batches refuse wide members; more
    than 32,767 per vertex is refused at creation."""
    inst = _weighted_hub()
    h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
    b = pg.pamc_batch_create(0)
    try:
        with pytest.raises(pg.PamcError) as e:
            pg.pamc_init(h, kind=1, R=8, steps=2)
        assert e.value.status == 4
        pg.pamc_init(h, R=8, steps=2)
        with pytest.raises(pg.PamcError):
            pg.pamc_batch_add(b, h)
    finally:
        pg.pamc_batch_destroy(b)
        pg.pamc_destroy(h)
    n = 300                                   # a vertex with 299 couplings of 127: 37,973 > 32,767
    big = W.csr_from_edges(n, np.zeros(n - 1, dtype=np.int64), np.arange(1, n), np.full(n - 1, 127), "star127")
    with pytest.raises(pg.PamcError) as e:
        pg.pamc_create_csr(big.n, big.row_ptr, big.col, big.w)
    assert e.value.status == 4


def _max_degree_graph(n, m, dmax, seed, weights=(-1, 1)):
    """A random graph with every degree <= dmax, some = dmax, weights drawn
    from the given values."""
    rng = np.random.default_rng(seed)
    deg = np.zeros(n, dtype=np.int64)
    pairs = set()
    while len(pairs) < m:
        a, b = (int(x) for x in rng.integers(0, n, size=2))
        if a == b or (min(a, b), max(a, b)) in pairs or deg[a] >= dmax or deg[b] >= dmax:
            continue
        pairs.add((min(a, b), max(a, b)))
        deg[a] += 1
        deg[b] += 1
    ei, ej = np.array(sorted(pairs)).T
    w = rng.choice(np.asarray(weights), size=len(ei))
    inst = W.csr_from_edges(n, ei, ej, w, f"maxdeg{dmax}")
    assert deg.max() == dmax
    return inst


def _half_row_ranges(inst):
    """Per vertex, sum |w| over its first eight nonzero couplings (CSR order:
    the ELL slots 0..7) and over the rest."""
    out = []
    for k in range(inst.n):
        w = inst.w[inst.row_ptr[k]:inst.row_ptr[k + 1]]
        w = np.abs(w[w != 0])
        out.append((int(w[:8].sum()), int(w[8:].sum())))
    return np.array(out)


@pytest.mark.parametrize("nib", ["1", "0"])
@pytest.mark.parametrize("rule", [0, 1])
def test_nibble_lanes(pg, monkeypatch, nib, rule):
    """Field ranges that fit 4-bit lanes run eight replicas per word: the
    fixed bias (range <= 7) on ELL rows of width 4 (torus) and 8 (degree 7),
    and the biased lanes with two half-row accumulators (each half-row's
    range <= 15) on widths 8, 12 and 16, +-1 and weighted couplings.  The
    oracle's results step after step with ragged populations (R not a
    multiple of 8), cluster moves and restarts, and with the lanes switched
    off."""
    monkeypatch.setenv("PAMC_SWEEP_NIBBLE", nib)
    cases = ((W.torus(18, 18, signed=True, seed=3), 13), (_max_degree_graph(400, 1100, 7, 4), 21),
             (_max_degree_graph(300, 700, 6, 5), 8), (_max_degree_graph(300, 900, 8, 6), 16),
             (_max_degree_graph(500, 2400, 12, 7), 19), (_max_degree_graph(600, 3600, 16, 8), 27),
             (_max_degree_graph(400, 1000, 7, 9, weights=(-2, -1, 1, 2)), 11),
             (_max_degree_graph(500, 2000, 16, 10, weights=(-2, -1, -1, 1, 1, 2)), 24))
    for inst, R in cases:
        half = _half_row_ranges(inst)
        assert half.max() <= 15, inst.name           # every case fits the biased lanes
        s = pg.Solver(inst.row_ptr, inst.col, inst.w)
        s.init(R=R, sweeps=3, steps=3, rule=rule, seed=4)
        assert pg.pamc_sweep_mode(s.h) == (17 if nib == "1" else 1), inst.name
        s.close()
        compare_run(pg, inst, 10, R=R, sweeps=3, beta0=0.2, beta1=3.0, rule=rule, stagnation=1, z_rst=7,
                    cooldown_tau=1, win_short=2, win_long=3, seed=4)


def test_nibble_lanes_limits(pg):
    """A half-row range of 16 (or a row wider than 16) keeps the byte lanes;
    15 takes the biased 4-bit lanes."""
    n = 40
    for wv, mode in ((2, 1), ((2, 2, 2, 2, 2, 2, 2, 1), 17)):
        ws = np.resize(np.asarray(wv), 8)
        inst = W.csr_from_edges(n, np.zeros(8, dtype=np.int64), np.arange(1, 9), ws, "star8")
        assert _half_row_ranges(inst).max() == int(ws.sum())
        s = pg.Solver(inst.row_ptr, inst.col, inst.w)
        s.init(R=16, sweeps=2, steps=3, seed=1)
        assert pg.pamc_sweep_mode(s.h) == mode, ws
        s.close()
        compare_run(pg, inst, 4, R=16, sweeps=2, beta0=0.2, beta1=2.0, seed=3)
    hub = W.csr_from_edges(n, np.zeros(17, dtype=np.int64), np.arange(1, 18), np.ones(17), "star17")
    s = pg.Solver(hub.row_ptr, hub.col, hub.w)
    s.init(R=16, sweeps=2, steps=3, seed=1)
    assert pg.pamc_sweep_mode(s.h) == 1
    s.close()


@pytest.mark.parametrize("rule", [0, 1])
def test_maximum_population(pg, rule):
    """R = 16,384, the largest population pamc_init takes (4,096 replica
    groups, 1,024 cluster-move targets), against the oracle step by step."""
    inst = W.torus(12, 12, signed=True, seed=7)
    ref, _ = compare_run(pg, inst, 6, R=16384, sweeps=2, beta0=0.3, beta1=3.0, rule=rule, stagnation=1, z_rst=0,
                         cooldown_tau=1, win_short=2, win_long=3, seed=5)
    assert ref.ctl()["ncm_flipped"] > 0


@pytest.mark.parametrize("R,extra", [(16385, dict(stagnation=1, n_top=3000)),
                                     (32768, dict(stagnation=1, rule=1)),
                                     (20001, dict(stagnation=1, n_top=16384, z_rst=5)),
                                     (65536, dict())])
def test_large_populations(pg, R, extra):
    """Populations above 16,384 (the population step in several kernels,
    prefix sums in device memory, NCM targets by radix select) against the
    oracle step by step: just above the threshold, ragged sizes, the largest
    NCM target count, both rules, a restart."""
    inst = W.torus(8, 8, signed=True, seed=11)
    params = dict(sweeps=2, beta0=0.3, beta1=3.0, win_short=2, win_long=3, cooldown_tau=1, seed=13)
    params.update(extra)
    ref, _ = compare_run(pg, inst, 7, R=R, **params)
    if params.get("stagnation"):
        assert ref.ctl()["ncm_flipped"] > 0


def test_large_population_limits(pg):
    inst = W.torus(8, 8, signed=True, seed=11)
    h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
    with pytest.raises(pg.PamcError) as e:       # too many NCM targets for the one-CTA sort
        pg.pamc_init(h, R=40000, steps=3, stagnation=1, n_top=16385)
    assert e.value.status == pg.STATUS_CODES["PAMC_ERR_RANGE"]
    with pytest.raises(pg.PamcError) as e:
        pg.pamc_init(h, R=(1 << 20) + 1, steps=3)
    assert e.value.status == pg.STATUS_CODES["PAMC_ERR_RANGE"]
    pg.pamc_init(h, R=40000, steps=3, stagnation=0, n_top=16385)   # no cluster moves: no limit on n_top
    pg.pamc_destroy(h)


def test_degenerate_sizes_other_placements(pg, monkeypatch):
    """One vertex, one replica, zero sweeps, with the spin words in device
    memory and with 16-bit field lanes."""
    one = W.csr_from_edges(1, np.zeros(0), np.zeros(0), np.zeros(0), "one")
    monkeypatch.setenv("PAMC_SWEEP_GLOBAL", "1")
    compare_run(pg, one, 3, R=3, sweeps=2)
    inst = W.gnm(50, 80, signed=True, seed=3)
    compare_run(pg, inst, 4, R=1, sweeps=1)
    compare_run(pg, inst, 3, R=8, sweeps=0)
    monkeypatch.delenv("PAMC_SWEEP_GLOBAL")
    pair = W.csr_from_edges(2, np.array([0]), np.array([1]), np.array([127]), "pair127")
    star = W.csr_from_edges(3, np.array([0, 0]), np.array([1, 2]), np.array([127, -100]), "star227")
    for g in (pair, star):
        compare_run(pg, g, 4, R=5, sweeps=2, beta0=0.001, beta1=0.05)
