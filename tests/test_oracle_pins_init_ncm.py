"""Pins of the oracle's initial population, its restart re-draw and its choice
of cluster-move targets, against facts fixed outside the oracle.

* Algorithm 1's initialisation draws every spin (Ising) or label (Potts)
  uniformly and independently.  The population is checked for balance per
  site and per replica (chi-square) and for pairwise independence of
  replicas that share a random call, replicas that do not, and neighbouring
  sites (2x2 or KxK contingency chi-square).
* A restart that resets the system (Sec. II, reset every 400 iterations)
  draws a population that is again uniform, is independent of the first
  one, and differs from it; with re-initialisation off, the population is
  kept as it was.
* The cluster move goes to "the n top configurations" of Algorithm 1: the
  n_top replicas of lowest energy (highest cut), ties to the lower slot.  A
  population of hand-built energy ties shows that exactly those replicas,
  and only those, change, and that the others stay bit for bit.

No GPU is needed.
"""
import numpy as np
import pytest
from scipy.stats import chi2 as chi2_dist

import oracle
import workloads as W

P_MIN = 1e-4     # p-value floor of every uniformity / independence test


def _initial(inst, **params):
    run = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, steps=4, **params)
    s = run.spins()
    run.close()
    return s


def _chi2_uniform(counts):
    """p-value of the counts under equal cell probabilities."""
    counts = np.asarray(counts, dtype=np.float64).ravel()
    exp = counts.sum() / counts.size
    stat = float(((counts - exp) ** 2 / exp).sum())
    return float(chi2_dist.sf(stat, counts.size - 1))


def _balance_pvalues(x, levels):
    """Chi-square p-values of label balance per site (columns) and per replica
    (rows), each summed over all sites / replicas (the sum of independent
    chi-square statistics is chi-square with the summed degrees of freedom)."""
    R, n = x.shape
    out = []
    for axis, m in ((0, R), (1, n)):
        stat, dof = 0.0, 0
        counts = np.stack([(x == v).sum(axis=axis) for v in levels], axis=-1).astype(np.float64)
        exp = m / len(levels)
        stat = float(((counts - exp) ** 2 / exp).sum())
        dof = counts.shape[0] * (len(levels) - 1)
        out.append(float(chi2_dist.sf(stat, dof)))
    return out


def _pair_pvalue(a, b, levels):
    """Chi-square p-value of the joint label counts of paired samples (a, b)
    against independence with uniform marginals (every cell 1/|levels|^2)."""
    L = len(levels)
    idx = {v: i for i, v in enumerate(levels)}
    ia = np.vectorize(idx.get)(a.ravel())
    ib = np.vectorize(idx.get)(b.ravel())
    return _chi2_uniform(np.bincount(ia * L + ib, minlength=L * L))


def _independence_pvalues(x, levels):
    """Replicas r, r+1 (words of one Philox call), r, r+4 (different calls),
    r, r+5, and neighbouring sites i, i+1."""
    return [_pair_pvalue(x[0:-1:2], x[1::2], levels),
            _pair_pvalue(x[:-4], x[4:], levels),
            _pair_pvalue(x[:-5], x[5:], levels),
            _pair_pvalue(x[:, :-1], x[:, 1:], levels)]


def test_initial_ising_population_uniform_and_independent():
    inst = W.gnm(300, 600, signed=True, seed=3)
    s = _initial(inst, R=1024, seed=17)
    assert set(np.unique(s).tolist()) == {-1, 1}
    for p in _balance_pvalues(s, (-1, 1)) + _independence_pvalues(s, (-1, 1)):
        assert p > P_MIN, p
    # a second seed gives an unrelated population
    s2 = _initial(inst, R=1024, seed=18)
    agree = float((s == s2).mean())
    assert abs(agree - 0.5) < 5 * 0.5 / np.sqrt(s.size)


@pytest.mark.parametrize("K,rule", [(3, 0), (5, 2), (8, 2)])
def test_initial_potts_labels_uniform_and_independent(K, rule):
    inst = W.gnm(200, 500, signed=False, seed=4)
    s = _initial(inst, kind=1, rule=rule, K=K, R=512, seed=5)
    levels = tuple(range(K))
    assert s.min() >= 0 and s.max() < K
    for p in _balance_pvalues(s, levels) + _independence_pvalues(s, levels):
        assert p > P_MIN, p


@pytest.mark.parametrize("kind", [0, 1])
def test_restart_redraws_an_independent_population(kind):
    """No sweeps and no resampling, so only a restart can change the
    population.  z_rst = 3: the third iteration restarts.  With
    re-initialisation the population after it is a fresh uniform draw
    unrelated to the first one (agreement 1/2 for spins, 1/3 for labels);
    without it the population is the first one, bit for bit."""
    inst = W.gnm(250, 700, signed=True, seed=6)
    params = dict(kind=kind, R=512, sweeps=0, steps=10, z_rst=3, resample=0, seed=21)
    levels = (-1, 1) if kind == 0 else (0, 1, 2)
    for reinit in (1, 0):
        run = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, restart_reinit=reinit, **params)
        s0 = run.spins()
        run.step(2)
        np.testing.assert_array_equal(run.spins(), s0)        # nothing moves before the restart
        run.step(1)
        assert run.ctl()["cycle"] == 1
        s1 = run.spins()
        E1 = run.energy()
        J = (-inst.w).astype(np.int32)
        efn = oracle.energy_ising if kind == 0 else oracle.energy_potts
        for r in range(0, params["R"], 37):
            assert E1[r] == efn(inst.row_ptr, inst.col, J, s1[r])
        if not reinit:
            np.testing.assert_array_equal(s1, s0)
            run.close()
            continue
        agree = float((s1 == s0).mean())
        p_agree = 1.0 / len(levels)
        sd = np.sqrt(p_agree * (1 - p_agree) / s0.size)
        assert abs(agree - p_agree) < 5 * sd, agree
        for p in _balance_pvalues(s1, levels) + _independence_pvalues(s1, levels):
            assert p > P_MIN, p
        # the re-drawn population is independent of the first, site by site
        assert _pair_pvalue(s0, s1, levels) > P_MIN
        # a second restart draws yet another population
        run.step(3)
        assert run.ctl()["cycle"] == 2
        s2 = run.spins()
        assert abs(float((s2 == s1).mean()) - p_agree) < 5 * sd
        run.close()


# ---------------------------------------------------------------- NCM targets
def _fields(inst, s):
    n = inst.n
    h = np.zeros(n, dtype=np.int64)
    J = -inst.w.astype(np.int64)
    for k in range(n):
        sl = slice(inst.row_ptr[k], inst.row_ptr[k + 1])
        h[k] = int((J[sl] * s[inst.col[sl]]).sum())
    return h


def _tied_population(inst, nbase, rng):
    """nbase configurations of distinct energies, each with iso-sites, and
    their global flips (same energy, same iso-sites): replica k holds base k,
    replica k + nbase its flip, so every energy occurs exactly twice."""
    J = (-inst.w).astype(np.int32)
    bases, energies = [], set()
    while len(bases) < nbase:
        s = rng.choice(np.array([-1, 1], dtype=np.int8), size=inst.n)
        e = oracle.energy_ising(inst.row_ptr, inst.col, J, s)
        if e in energies or not (_fields(inst, s) == 0).any():
            continue
        energies.add(e)
        bases.append(s)
    pop = np.concatenate([np.stack(bases), -np.stack(bases)]).astype(np.int8)
    E = np.array([oracle.energy_ising(inst.row_ptr, inst.col, J, x) for x in pop], dtype=np.int64)
    return pop, E


@pytest.mark.parametrize("n_top,seed", [(5, 1), (1, 2), (6, 3), (9, 4)])
def test_ncm_targets_are_the_lowest_energy_replicas_ties_to_lower_slot(n_top, seed):
    """Constant M* (no sweeps, no resampling) stagnates both windows of
    lengths 2 and 3 after three iterations; the controller arms the cluster
    move and the fourth iteration applies it.  Energies come in tied pairs
    (a configuration and its global flip), ordered by construction, so the
    expected targets are known without sorting: the pairs of the lowest
    energies, and where n_top splits a pair, its lower slot only."""
    inst = W.torus(10, 10, signed=True, seed=seed)
    nbase = 8
    rng = np.random.default_rng(seed)
    pop, E = _tied_population(inst, nbase, rng)
    R = 2 * nbase
    run = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, R=R, sweeps=0, steps=50, stagnation=1,
                           resample=0, z_rst=0, win_short=2, win_long=3, max_distinct_short=3,
                           max_distinct_long=5, cooldown_tau=100, n_top=n_top, mis_trials=4, seed=seed)
    run.set_spins(pop)
    np.testing.assert_array_equal(run.energy(), E)
    run.step(3)
    assert run.ctl()["enable_cm"] == 1 and run.ctl()["ncm_last"] == 0
    run.step(1)
    assert run.ctl()["ncm_last"] == 1
    after = run.spins()
    changed = {r for r in range(R) if not np.array_equal(after[r], pop[r])}
    # base k sits at slots k and k + nbase; bases ranked by energy
    rank = sorted(range(nbase), key=lambda k: int(E[k]))
    want = []
    for k in rank:
        for slot in (k, k + nbase):         # lower slot first within a tie
            if len(want) < n_top:
                want.append(slot)
    assert changed == set(want), (sorted(changed), sorted(want))
    for r in set(range(R)) - changed:
        np.testing.assert_array_equal(after[r], pop[r])
    np.testing.assert_array_equal(run.energy(), E)            # the move keeps every energy
    run.close()
