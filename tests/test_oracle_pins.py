"""Pins of the CPU oracle against facts fixed outside it.

Each test checks the oracle against something other than itself: published
known-answer vectors, libm, closed forms from the paper's equations, exhaustive
enumeration on tiny instances, the exact Boltzmann distribution, or invariants
the method guarantees.  No GPU is needed.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TWO32 = 1 << 32


# ------------------------------------------------------------------ Philox
def test_philox_known_answers():
    """Random123's published Philox4x32-10 vectors (SC'11 generator)."""
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        vals = [int(x, 16) for x in row]
        ctr, key, want = vals[0:4], vals[4:6], vals[6:10]
        got = oracle.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == want


# ------------------------------------------------------------------ det_exp
def test_det_exp_within_one_ulp_of_libm():
    """One million points over the whole unflushed range [-707, 709], the
    small-|x| band and the range the weights and thresholds use."""
    rng = np.random.default_rng(7)
    xs = np.concatenate([rng.uniform(-707, 709, 600000), rng.uniform(-2, 2, 200000),
                         rng.uniform(-60, 0, 200000)])
    f = oracle.lib().orc_det_exp
    worst = 0.0
    for x in xs.tolist():
        a, b = f(x), math.exp(x)
        worst = max(worst, abs(a - b) / math.ulp(b))
    assert worst <= 1.0


def test_det_exp_special_values_and_monotone():
    assert oracle.det_exp(0.0) == 1.0
    assert oracle.det_exp(-708.0) == 0.0
    assert math.isinf(oracle.det_exp(710.0))
    grid = np.linspace(-30, 30, 60001)
    vals = np.array([oracle.det_exp(x) for x in grid])
    assert np.all(np.diff(vals) >= 0)


def test_round_nonneg():
    for x, want in [(0.0, 0), (0.49999999999999994, 0), (0.5, 1), (1.5, 2), (2.5, 3),
                    (4294967295.5, 4294967296), (4294967296.0, 4294967296), (7.25, 7)]:
        assert oracle.round_nonneg(x) == want


# ------------------------------------------------------------------ thresholds
@pytest.mark.parametrize("beta", [0.01, 0.1, 0.7, 3.0])
def test_heatbath_threshold_is_eq4(beta):
    """T(h)/2^32 = (1 + tanh(beta h))/2, the Eq. 4 probability of s=+1."""
    for h in range(-60, 61):
        T = oracle.thr_heatbath(beta, h)
        exact = TWO32 * (1.0 + math.tanh(beta * h)) / 2.0
        assert abs(T - exact) <= 1.0 + 1e-6 * exact
        assert 0 <= T <= TWO32
    assert oracle.thr_heatbath(beta, 0) == TWO32 // 2


@pytest.mark.parametrize("beta", [0.05, 0.5, 2.0])
def test_metropolis_threshold(beta):
    for dE in range(-20, 41):
        T = oracle.thr_metropolis(beta, dE)
        if dE <= 0:
            assert T == TWO32
        else:
            assert abs(T - TWO32 * math.exp(-beta * dE)) <= 1.0 + 1e-9 * TWO32


@pytest.mark.parametrize("beta", [0.1, 0.9, 2.5])
def test_cascaded_sampler_reproduces_softmax(beta):
    """Suppl. S3: P(0)=T1, P(1)=(1-T1)T2, P(2)=(1-T1)(1-T2) equal the Eq. 8 softmax."""
    rng = np.random.default_rng(3)
    for _ in range(300):
        syn = rng.integers(-12, 1, size=3)
        z = np.exp(beta * syn.astype(np.float64))
        soft = z / z.sum()
        t1 = oracle.thr_potts_b1(beta, syn[1] - syn[0], syn[2] - syn[0]) / TWO32
        t2 = oracle.thr_potts_b2(beta, syn[2] - syn[1]) / TWO32
        got = np.array([t1, (1 - t1) * t2, (1 - t1) * (1 - t2)])
        assert np.allclose(got, soft, atol=4.0 / TWO32, rtol=0)


# ------------------------------------------------------------------ permutation
def test_permutation_is_uniform_and_shared_order():
    n = 7
    counts = np.zeros((n, n))
    for t in range(600):
        for sw in range(5):
            p = oracle.permutation(n, 11, t, sw)
            assert sorted(p.tolist()) == list(range(n))
            counts[p, np.arange(n)] += 1
    from scipy.stats import chisquare
    assert chisquare(counts.ravel()).pvalue > 1e-4
    assert not np.array_equal(oracle.permutation(50, 1, 0, 0), oracle.permutation(50, 1, 0, 1))
    assert np.array_equal(oracle.permutation(50, 1, 3, 2), oracle.permutation(50, 1, 3, 2))


# ------------------------------------------------------------------ resampling
def _tau(E, delta, escale=1.0):
    E = np.asarray(E, dtype=np.float64)
    x = -delta * escale * E          # Eq. 1 weight exp(-(beta_{i+1}-beta_i) E_j)
    w = np.exp(x - x.max())
    return len(E) * w / w.sum()


def test_resample_conserves_population_and_rounds_tau():
    rng = np.random.default_rng(5)
    for trial in range(200):
        R = int(rng.integers(1, 300))
        E = rng.integers(-2000, 2000, size=R)
        delta = float(rng.choice([0.02, -0.02, 0.3, 0.0005]))
        par, cnt = oracle.resample(E, delta, 1.0, 9, trial)
        assert cnt.sum() == R
        assert np.all(np.diff(par) >= 0)
        assert np.array_equal(np.bincount(par, minlength=R), cnt)
        tau = _tau(E, delta)
        assert np.all(cnt >= np.floor(tau - 1e-6)) and np.all(cnt <= np.ceil(tau + 1e-6))


def test_resample_zero_delta_is_identity():
    E = np.array([5, -3, 100, 7, 7, 0], dtype=np.int64)
    par, cnt = oracle.resample(E, 0.0, 1.0, 1, 4)
    assert par.tolist() == list(range(6)) and cnt.tolist() == [1] * 6


def test_resample_expected_copies_equal_tau():
    """Eq. 1-2 read as expected copy numbers summing to R."""
    E = np.array([0, 1, 2, 3, 5, 8, 13, 21], dtype=np.int64)
    delta = 0.15
    tot = np.zeros(8)
    T = 4000
    for t in range(T):
        _, cnt = oracle.resample(E, delta, 1.0, 21, t)
        tot += cnt
    assert np.allclose(tot / T, _tau(E, delta), atol=0.03)


# ------------------------------------------------------------------ energies
def _dense_J(inst):
    J = np.zeros((inst.n, inst.n), dtype=np.int64)
    for i in range(inst.n):
        for e in range(inst.row_ptr[i], inst.row_ptr[i + 1]):
            J[i, inst.col[e]] = -inst.w[e]
    return J


def test_energy_and_cut_identity():
    inst = W.erdos_renyi(40, 0.2, signed=True, seed=2)
    J = _dense_J(inst)
    Jcsr = -inst.w
    Wsum = int(np.triu(-J).sum())
    rng = np.random.default_rng(0)
    for _ in range(20):
        s = rng.choice([-1, 1], size=inst.n).astype(np.int8)
        E = oracle.energy_ising(inst.row_ptr, inst.col, Jcsr, s)
        assert E == int(-0.5 * s.astype(np.int64) @ J @ s.astype(np.int64))
        cut = int(sum((-J[i, j]) for i in range(inst.n) for j in range(i + 1, inst.n)
                      if J[i, j] != 0 and s[i] != s[j]))
        assert cut == (Wsum - E) // 2 and (Wsum - E) % 2 == 0
        lab = rng.integers(0, 3, size=inst.n).astype(np.int8)
        Ep = oracle.energy_potts(inst.row_ptr, inst.col, Jcsr, lab)
        same = (lab[:, None] == lab[None, :]).astype(np.int64)
        assert Ep == int(-np.triu(J * (2 * same - 1), 1).sum())
        cut3 = int(sum((-J[i, j]) for i in range(inst.n) for j in range(i + 1, inst.n)
                       if J[i, j] != 0 and lab[i] != lab[j]))
        assert cut3 == (Wsum - Ep) // 2


@pytest.mark.parametrize("kind,rule", [(0, 0), (0, 1), (1, 0)])
def test_incremental_fields_match_recompute(kind, rule):
    inst = W.gnm(60, 150, signed=True, seed=4)
    run = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, kind=kind, rule=rule, R=12, sweeps=3,
                           steps=8, beta0=0.2, beta1=2.0)
    J = _dense_J(inst)
    for _ in range(8):
        run.step(1)
        s = run.spins().astype(np.int64)
        f = run.fields()
        E = run.energy()
        if kind == 0:
            assert np.array_equal(f, s @ J.T)
            assert np.array_equal(E, (-0.5 * np.einsum("ri,ij,rj->r", s, J, s)).astype(np.int64))
        else:
            onehot = np.stack([(s == c).astype(np.int64) for c in range(3)], axis=-1)
            assert np.array_equal(f, np.einsum("ij,rjc->ric", J, onehot))
            for r in range(12):
                assert E[r] == oracle.energy_potts(inst.row_ptr, inst.col, -inst.w, s[r].astype(np.int8))


# ------------------------------------------------------------------ brute force optimum
def _brute_maxcut(inst):
    n = inst.n
    states = ((np.arange(1 << n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int8)
    cut = np.zeros(1 << n, dtype=np.int64)
    for i in range(n):
        for e in range(inst.row_ptr[i], inst.row_ptr[i + 1]):
            j = inst.col[e]
            if i < j:
                cut += inst.w[e] * (states[:, i] != states[:, j])
    return int(cut.max())


def _brute_max3cut(inst):
    n = inst.n
    states = np.array(list(itertools.product(range(3), repeat=n)), dtype=np.int8)
    cut = np.zeros(states.shape[0], dtype=np.int64)
    for i in range(n):
        for e in range(inst.row_ptr[i], inst.row_ptr[i + 1]):
            j = inst.col[e]
            if i < j:
                cut += inst.w[e] * (states[:, i] != states[:, j])
    return int(cut.max())


@pytest.mark.parametrize("seed,signed", [(0, False), (1, True), (2, True)])
def test_pamc_finds_brute_force_maxcut(seed, signed):
    inst = W.erdos_renyi(16, 0.4, signed=signed, seed=seed)
    opt = _brute_maxcut(inst)
    run = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, R=64, sweeps=2, steps=40, beta0=0.1,
                           beta1=3.0, seed=seed)
    run.step(40)
    m, best = run.best()
    assert m == opt
    cut = sum(inst.w[e] for i in range(inst.n) for e in range(inst.row_ptr[i], inst.row_ptr[i + 1])
              if i < inst.col[e] and best[i] != best[inst.col[e]])
    assert cut == m and best[0] == 1


def test_potts_finds_brute_force_max3cut():
    inst = W.erdos_renyi(9, 0.6, signed=False, seed=5)
    opt = _brute_max3cut(inst)
    run = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, kind=1, R=64, sweeps=2, steps=40,
                           beta0=0.1, beta1=3.0, seed=3)
    run.step(40)
    m, best = run.best()
    assert m == opt
    assert best[0] == 0


def test_target_cut_stops_early():
    inst = W.erdos_renyi(16, 0.4, signed=False, seed=0)
    opt = _brute_maxcut(inst)
    run = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, R=64, sweeps=2, steps=400, beta0=0.1,
                           beta1=3.0, target_cut=opt)
    ran = run.step(400)
    assert ran < 400 and run.ctl()["done"] == 1 and run.best()[0] == opt


# ------------------------------------------------------------------ Boltzmann sampling
def _chi2_pvalue(obs, p):
    from scipy.stats import chi2
    exp = p * obs.sum()
    keep = exp > 5
    stat = float((((obs - exp) ** 2) / np.where(exp > 0, exp, 1))[keep].sum())
    return chi2.sf(stat, keep.sum() - 1)


@pytest.mark.parametrize("rule", [0, 1])
def test_fixed_beta_sweeps_sample_boltzmann_ising(rule):
    """Eq. 4 (heat-bath) and Metropolis leave exp(-beta H) invariant."""
    inst = W.erdos_renyi(6, 0.7, signed=True, seed=8)
    beta = 0.45
    n = inst.n
    run = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, rule=rule, R=512, sweeps=1, steps=60,
                           beta0=beta, beta1=beta, resample=0, seed=17)
    obs = np.zeros(1 << n)
    for step in range(60):
        run.step(1)
        if step >= 10 and step % 2 == 0:
            s = run.spins()
            code = ((s > 0).astype(np.int64) << np.arange(n)).sum(axis=1)
            obs += np.bincount(code, minlength=1 << n)
    states = np.where(((np.arange(1 << n)[:, None] >> np.arange(n)) & 1) == 1, 1, -1).astype(np.int8)
    E = np.array([oracle.energy_ising(inst.row_ptr, inst.col, -inst.w, s) for s in states], dtype=np.float64)
    p = np.exp(-beta * E)
    p /= p.sum()
    assert _chi2_pvalue(obs, p) > 1e-4
    # a wrong temperature is rejected by the same statistic
    q = np.exp(-2 * beta * E)
    q /= q.sum()
    assert _chi2_pvalue(obs, q) < 1e-6


def test_fixed_beta_sweeps_sample_potts():
    """Cascaded sampler at Eq. 8's beta samples exp(-(beta/2) E) of Eq. 6."""
    inst = W.erdos_renyi(5, 0.8, signed=True, seed=6)
    beta = 0.8
    n = inst.n
    run = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, kind=1, R=1024, sweeps=1, steps=50,
                           beta0=beta, beta1=beta, resample=0, seed=23)
    obs = np.zeros(3 ** n)
    for step in range(50):
        run.step(1)
        if step >= 10 and step % 2 == 0:
            s = run.spins().astype(np.int64)
            code = (s * (3 ** np.arange(n))).sum(axis=1)
            obs += np.bincount(code, minlength=3 ** n)
    states = np.array(list(itertools.product(range(3), repeat=n)), dtype=np.int8)[:, ::-1]
    E = np.array([oracle.energy_potts(inst.row_ptr, inst.col, -inst.w, np.ascontiguousarray(s))
                  for s in states], dtype=np.float64)
    p = np.exp(-0.5 * beta * E)
    p /= p.sum()
    assert _chi2_pvalue(obs, p) > 1e-4
    q = np.exp(-beta * E)
    q /= q.sum()
    assert _chi2_pvalue(obs, q) < 1e-6


# ------------------------------------------------------------------ NCM
def test_ncm_preserves_energy_and_builds_maximal_independent_iso_set():
    inst = W.torus(12, 12, signed=True, seed=1)
    J = _dense_J(inst)
    rng = np.random.default_rng(2)
    for r in range(30):
        s = rng.choice([-1, 1], size=inst.n).astype(np.int8)
        h = (J @ s.astype(np.int64)).astype(np.int32)
        iso = set(np.nonzero(h == 0)[0].tolist())
        E0 = oracle.energy_ising(inst.row_ptr, inst.col, -inst.w, s)
        s1, h1 = s.copy(), h.copy()
        k = oracle.ncm_replica(inst.row_ptr, inst.col, -inst.w, s1, h1, 4, 99, 3, r)
        flipped = set(np.nonzero(s1 != s)[0].tolist())
        assert len(flipped) == k and flipped <= iso
        assert all(J[a, b] == 0 for a in flipped for b in flipped if a != b)
        assert all(any(J[a, b] != 0 for b in flipped) for a in iso - flipped)
        assert oracle.energy_ising(inst.row_ptr, inst.col, -inst.w, s1) == E0
        assert np.array_equal(h1, (J @ s1.astype(np.int64)).astype(np.int32))


def test_ncm_on_dense_flips_at_most_one_site():
    inst = W.dense_csr(24, seed=3)
    J = _dense_J(inst)
    rng = np.random.default_rng(4)
    for r in range(40):
        s = rng.choice([-1, 1], size=inst.n).astype(np.int8)
        h = (J @ s.astype(np.int64)).astype(np.int32)
        s1 = s.copy()
        k = oracle.ncm_replica(inst.row_ptr, inst.col, -inst.w, s1, h.copy(), 4, 5, 0, r)
        assert k == (1 if (h == 0).any() else 0)


# ------------------------------------------------------------------ controller
def _ctl(**kw):
    return oracle.Controller(stagnation=1, beta0=0.1, beta1=2.1, steps=101, z_rst=0, **kw)


def test_controller_keeps_cooling_while_progressing():
    c = _ctl()
    beta = 0.1
    for m in range(60):
        assert not c.update(m)
        beta = beta + 0.02
        st = c.state()
        assert st["delta"] == pytest.approx(0.02) and st["enable_cm"] == 0
        assert st["beta"] == beta


def test_controller_strong_stagnation_reheats_and_arms_ncm():
    c = _ctl()
    beta = 0.1
    for i in range(39):
        c.update(7)
        beta = beta + 0.02
    assert c.state()["enable_cm"] == 0 and c.state()["beta"] == beta
    c.update(7)                      # 40th entry: both windows hold one value
    st = c.state()
    assert st["enable_cm"] == 1
    assert st["beta"] == 0.8 * beta + 0.02
    assert st["delta"] == pytest.approx(0.02)


def test_controller_mild_stagnation_reverses_beta():
    c = _ctl()
    seq = list(range(1, 16)) + [15] * 25      # 40 entries: last 25 one value, last 40 fifteen
    beta = 0.1
    for m in seq[:-1]:
        c.update(m)
        beta = beta + 0.02
    c.update(seq[-1])
    st = c.state()
    assert st["enable_cm"] == 0
    assert st["delta"] == pytest.approx(-0.02)
    assert st["beta"] == pytest.approx(beta - 0.02)


def test_controller_restart_resets_schedule():
    c = oracle.Controller(stagnation=1, beta0=0.1, beta1=2.1, steps=101, z_rst=5)
    flags = [c.update(m) for m in range(5)]
    assert flags == [False, False, False, False, True]
    st = c.state()
    assert st["z"] == 1 and st["cycle"] == 1 and st["beta"] == 0.1 and st["hist_len"] == 0


# ------------------------------------------------------------------ SA baseline
def test_without_resampling_replicas_are_independent_chains():
    inst = W.gnm(30, 60, signed=True, seed=1)
    a = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, R=4, sweeps=2, steps=6, resample=0)
    b = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, R=9, sweeps=2, steps=6, resample=0)
    a.step(6)
    b.step(6)
    assert np.array_equal(a.spins(), b.spins()[:4])


def test_augmented_run_invokes_ncm_and_preserves_energy():
    inst = W.torus(16, 16, signed=True, seed=2)
    run = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, R=32, sweeps=2, steps=150, beta0=0.5,
                           beta1=6.0, stagnation=1, z_rst=120, cooldown_tau=5)
    run.step(150)
    st = run.ctl()
    assert st["ncm_flipped"] > 0 and st["ncm_dE_max"] == 0 and st["cycle"] == 1


# ---------------------------------------------------------------- diagnostics
def test_hamming_hand_example():
    """Three replicas of four spins: d(s0,s1)=1, d(s0,s2)=4 -> 0 (complement),
    d(s1,s2)=3 -> 1; histogram [1, 2, 0], sum 2, mean 2 / (3 pairs * 4)."""
    s = np.array([[1, 1, 1, 1], [1, -1, 1, 1], [-1, -1, -1, -1]], dtype=np.int8)
    hist, total = oracle.hamming_counts(s)
    assert hist.tolist() == [1, 2, 0]
    assert total == 2


def test_hamming_symmetries():
    rng = np.random.default_rng(5)
    s = np.where(rng.random((7, 11)) < 0.5, 1, -1).astype(np.int8)
    hist, total = oracle.hamming_counts(s)
    assert hist.sum() == 7 * 6 // 2
    assert total == int((np.arange(hist.size) * hist).sum())
    # flipping a whole replica or permuting the spins changes nothing
    s2 = s.copy()
    s2[3] = -s2[3]
    perm = rng.permutation(11)
    for other in (s2, s[:, perm], s[::-1]):
        h2, t2 = oracle.hamming_counts(other)
        assert h2.tolist() == hist.tolist() and t2 == total


def test_hamming_distribution_of_independent_pairs():
    """Independent uniform replicas: d ~ Binomial(n, 1/2), so dc = min(d, n-d)
    has P(k) = 2 C(n,k) / 2^n for k < n/2 and C(n, n/2) / 2^n at k = n/2."""
    n, trials = 6, 20000
    rng = np.random.default_rng(9)
    counts = np.zeros(n // 2 + 1)
    for _ in range(trials):
        s = np.where(rng.random((2, n)) < 0.5, 1, -1).astype(np.int8)
        counts += oracle.hamming_counts(s)[0]
    p = np.array([2 * math.comb(n, k) for k in range(n // 2)] + [math.comb(n, n // 2)]) / 2 ** n
    chi2 = float(((counts - trials * p) ** 2 / (trials * p)).sum())
    assert chi2 < 16.3   # 3 degrees of freedom, p = 0.001


def test_lineage_composition():
    fam = np.arange(6)
    fam = oracle.lineage_step(fam, [0, 0, 2, 3, 3, 3])
    assert fam.tolist() == [0, 0, 2, 3, 3, 3]
    fam = oracle.lineage_step(fam, [1, 1, 1, 4, 5, 5])
    assert fam.tolist() == [0, 0, 0, 3, 3, 3]
    assert oracle.lineage_step(fam, [0] * 6, reinitialised=True).tolist() == list(range(6))


# ---------------------------------------------------------------- softmax Potts
def test_softmax_pick_gamma_zero_is_argmax():
    """gamma = 0: the label with the largest probability, i.e. the largest
    syn (softmax is monotone), the first one on ties."""
    rng = np.random.default_rng(11)
    for _ in range(300):
        K = int(rng.integers(2, 9))
        syn = rng.integers(-6, 7, size=K)
        u = rng.integers(0, 2 ** 32, size=K, dtype=np.uint64).astype(np.uint32)
        assert oracle.softmax_pick(syn, 0.7, 0.0, u) == int(np.argmax(syn))


def test_softmax_pick_two_labels_closed_form():
    """K = 2: label 0 wins iff U1 - U0 >= a = (P1 - P0) / gamma, and U1 - U0 is
    triangular on [-1, 1]: P(0) = (1 - a)^2 / 2 for a >= 0, 1 - (1 + a)^2 / 2
    for a < 0."""
    rng = np.random.default_rng(12)
    N = 40000
    for syn, beta, gamma in [((0, 2), 0.4, 1.0), ((3, -1), 0.25, 0.7), ((1, 1), 1.0, 1.0), ((0, 5), 0.3, 2.0)]:
        p1 = 1.0 / (1.0 + math.exp(beta * (syn[0] - syn[1])))
        a = (p1 - (1.0 - p1)) / gamma
        expect = (1 - a) ** 2 / 2 if a >= 0 else 1 - (1 + a) ** 2 / 2
        u = rng.integers(0, 2 ** 32, size=(N, 2), dtype=np.uint64).astype(np.uint32)
        zeros = sum(oracle.softmax_pick(syn, beta, gamma, u[i]) == 0 for i in range(N))
        sd = math.sqrt(expect * (1 - expect) / N)
        assert abs(zeros / N - expect) < 5 * sd + 1e-4, (syn, beta, gamma, zeros / N, expect)


def test_softmax_pick_large_noise_is_uniform():
    rng = np.random.default_rng(13)
    K, N = 5, 20000
    counts = np.zeros(K)
    syn = np.array([4, -2, 0, 1, 3])
    for i in range(N):
        u = rng.integers(0, 2 ** 32, size=K, dtype=np.uint64).astype(np.uint32)
        counts[oracle.softmax_pick(syn, 0.5, 1e6, u)] += 1
    chi2 = float(((counts - N / K) ** 2 / (N / K)).sum())
    assert chi2 < 18.5   # 4 degrees of freedom, p = 0.001


@pytest.mark.parametrize("K", [2, 3, 5, 8])
def test_softmax_potts_run_invariants(K):
    """A softmax Potts run keeps its incremental syn fields and energies equal
    to the definitions (Eq. 6-7) and labels in range; cut = (W - E)/2."""
    inst = W.gnm(60, 170, signed=True, seed=K)
    run = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, kind=1, rule=2, K=K, gamma=0.8, R=12, sweeps=2,
                           steps=6, seed=4)
    rp, col = inst.row_ptr, inst.col
    J = -inst.w
    for _ in range(6):
        run.step(1)
        s = run.spins()
        assert s.min() >= 0 and s.max() < K
        F = run.fields()
        E = run.energy()
        for r in range(run.R):
            syn = np.zeros((inst.n, K), dtype=np.int64)
            for k in range(inst.n):
                for e in range(rp[k], rp[k + 1]):
                    syn[k, s[r, col[e]]] += J[e]
            np.testing.assert_array_equal(F[r], syn)
            assert E[r] == oracle.energy_potts(rp, col, J.astype(np.int32), s[r])
    m, best = run.best()
    assert m == (run.weight_sum() - oracle.energy_potts(rp, col, J.astype(np.int32),
                                                        best.astype(np.int8))) // 2
    run.close()


def test_dense_sk_anneal_reaches_parisi_neighbourhood():
    """A loose physics pin for the fully connected +-1 instance (Sec. III.G):
    annealed ground-state energies of the Sherrington-Kirkpatrick model
    approach E / N^{3/2} = -0.7633 (Parisi) as N grows.  Four N=256 instances
    annealed by conventional PAMC land near it, and a run held hot does not
    (so a broken sampler or resampler fails the band)."""
    n = 256
    dens = []
    for sd in range(4):
        inst = W.dense_csr(n, seed=sd)
        run = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, R=64, sweeps=2, steps=300, beta0=0.01,
                               beta1=1.0, seed=0)
        run.step(300)
        m, best = run.best()
        e = run.weight_sum() - 2 * m
        J = -inst.w.astype(np.int64)
        s = best.astype(np.int64)
        assert e == -sum(J[q] * s[k] * s[inst.col[q]] for k in range(n)
                         for q in range(inst.row_ptr[k], inst.row_ptr[k + 1]) if inst.col[q] > k)
        dens.append(e / n ** 1.5)
        run.close()
    assert -0.80 <= float(np.mean(dens)) <= -0.72
    inst = W.dense_csr(n, seed=0)
    hot = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, R=64, sweeps=2, steps=300, beta0=0.001,
                           beta1=0.002, seed=0)
    hot.step(300)
    m, _ = hot.best()
    assert (hot.weight_sum() - 2 * m) / n ** 1.5 > -0.5
    hot.close()


def _weighted(n, p, wmax, seed):
    rng = np.random.default_rng(seed)
    ei, ej, w = [], [], []
    for i in range(n):
        for j in range(i + 1, n):
            if rng.random() < p:
                ei.append(i); ej.append(j); w.append(int(rng.integers(1, wmax + 1)) * int(rng.choice([-1, 1])))
    return W.csr_from_edges(n, np.array(ei), np.array(ej), np.array(w), f"weighted{wmax}_s{seed}")


@pytest.mark.parametrize("seed", [0, 1])
def test_pamc_finds_brute_force_maxcut_large_weights(seed):
    """Weights up to 100 in magnitude (field ranges far beyond a byte, the
    regime of the 16-bit-lane sweep): the annealer over a temperature range
    scaled to the weights reaches the exhaustive optimum, and the best
    configuration's cut is what it reports."""
    inst = _weighted(16, 0.5, 100, seed)
    H = max(int(np.abs(inst.w[inst.row_ptr[i]:inst.row_ptr[i + 1]]).sum()) for i in range(inst.n))
    assert H > 127
    opt = _brute_maxcut(inst)
    run = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, R=64, sweeps=2, steps=60, beta0=0.001,
                           beta1=0.05, seed=seed)
    run.step(60)
    m, best = run.best()
    assert m == opt
    cut = sum(inst.w[e] for i in range(inst.n) for e in range(inst.row_ptr[i], inst.row_ptr[i + 1])
              if i < inst.col[e] and best[i] != best[inst.col[e]])
    assert cut == m


def test_thresholds_saturate_exactly_at_large_fields():
    """Large |h| (up to 32,767): the heat-bath threshold is exactly 2^32 or 0
    once the Eq. 4 probability is within half a unit of 2^-32 of 1 or 0, and
    Metropolis accepts every downhill move and no move whose e^{-beta dE}
    rounds to 0; both stay within one unit of the closed forms everywhere."""
    for beta in (0.001, 0.05, 1.0):
        for h in (-32767, -5000, -300, -128, 128, 300, 5000, 32767):
            T = oracle.thr_heatbath(beta, h)
            exact = TWO32 * (1.0 + math.tanh(beta * h)) / 2.0
            assert abs(T - exact) <= 1.0 + 1e-6 * exact and 0 <= T <= TWO32
            if beta * h > 12:
                assert T == TWO32
            if beta * h < -12:
                assert T == 0
            M = oracle.thr_metropolis(beta, 2 * h)
            if h <= 0:
                assert M == TWO32
            else:
                assert abs(M - TWO32 * math.exp(-2 * beta * h)) <= 1.0
