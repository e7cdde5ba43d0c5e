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


@pytest.mark.parametrize("rule", [0, 1])
def test_dense_cold_rare_flips(pg, rule):
    """A cold anneal (few positions flip per block after the first steps),
    so most blocks take the path where the chains load the rows of their own
    replicas' flips of the previous block instead of a produced tile, and the
    update CTAs produce only the upper part of the block tile."""
    compare_dense(pg, 1024, 12, R=16, sweeps=2, beta0=0.5, beta1=3.0, rule=rule, seed=9, check_every=3)


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


def _exact_fields(torch, Jd, S, chunk=4096):
    """H = J S^T row block by row block with fp32 products on CUDA cores
    (exact: integer sums below 2^24, TF32 off)."""
    Sf = torch.from_numpy(S).cuda().float().T.contiguous()
    out = torch.empty((S.shape[0], Jd.shape[0]), dtype=torch.int64, device="cuda")
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for r0 in range(0, Jd.shape[0], chunk):
            out[:, r0:r0 + chunk] = (Jd[r0:r0 + chunk].float() @ Sf).round().long().T
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return out.cpu().numpy()


@pytest.mark.parametrize("n", [32768, 100000])
def test_dense_recompute_exact_at_large_fields(pg, n):
    """The tensor-core recompute H = J S is the exact integer field where it
    needs the most bits: replica 0 equals row 0 of J, so h_0 = n - 1 (up to
    99,999 = 17 bits), replica 1 equals minus row 7 (h_7 = -(n - 1)), replica
    2 is all +1 (row sums).  Every field is compared with an exact fp32
    product on CUDA cores, and the energies with the definition; then the run
    goes on from the set population and is checked again."""
    import torch
    R, seed = 8, 5
    wd = torch.empty((n, n), dtype=torch.int8, device="cuda")
    for r0 in range(0, n, 2000):
        wd[r0:r0 + 2000] = -W.dense_rows_torch(n, r0, min(n, r0 + 2000), seed, device="cuda")
    h = pg.pamc_create_dense(n, wd)
    try:
        pg.pamc_init(h, R=R, sweeps=1, steps=4, seed=1)
        Jd = wd.neg_()                                    # J = -w, reusing the buffer
        rng = np.random.default_rng(0)
        S = np.where(rng.random((R, n)) < 0.5, 1, -1).astype(np.int8)
        S[0] = np.where(Jd[0].cpu().numpy() >= 0, 1, -1)
        S[1] = -np.where(Jd[7].cpu().numpy() >= 0, 1, -1)
        S[2] = 1
        pg.pamc_set_population(h, S)
        H = pg.pamc_fields(h, R, n)
        ref = _exact_fields(torch, Jd, S)
        assert H[0, 0] == n - 1 and H[1, 7] == -(n - 1)
        np.testing.assert_array_equal(H, ref)
        _, E, _, _ = pg.pamc_state(h, R, n)
        np.testing.assert_array_equal(E, -(S.astype(np.int64) * ref).sum(axis=1) // 2)
        pg.pamc_step(h, 2)
        spins, E2, _, _ = pg.pamc_state(h, R, n)
        H2 = pg.pamc_fields(h, R, n)
        ref2 = _exact_fields(torch, Jd, spins)
        np.testing.assert_array_equal(H2, ref2)
        np.testing.assert_array_equal(E2, -(spins.astype(np.int64) * ref2).sum(axis=1) // 2)
    finally:
        pg.pamc_destroy(h)


@pytest.mark.parametrize("n", [256, 1000])
def test_dense_rows_gathered(pg, n):
    """pamc_dense_rows counts, per sweep position, whether some replica's spin
    turned over at its visit (the rows the field update needs).  With one
    sweep per step every vertex is visited once, so the count is the number of
    vertices whose value after the sweep differs, in some replica, from the
    resampled population before it (oracle spins and parents); positions are
    n per step."""
    w, inst = dense_pair(n, 4)
    params = dict(R=12, sweeps=1, steps=6, beta0=0.05, beta1=2.0, seed=3)
    ref = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **params)
    h = pg.pamc_create_dense(n, w)
    try:
        pg.pamc_init(h, **params)
        want = 0
        prev = ref.spins()
        for _ in range(params["steps"]):
            pg.pamc_step(h, 1)
            ref.step(1)
            par, _ = ref.parents()
            cur = ref.spins()
            want += int((cur != prev[par]).any(axis=0).sum())
            prev = cur
        rows, positions = pg.pamc_dense_rows(h)
        assert positions == n * params["steps"]
        assert rows == want
    finally:
        pg.pamc_destroy(h)
    small = W.torus(6, 6, signed=True, seed=1)
    hs = pg.pamc_create_csr(small.n, small.row_ptr, small.col, small.w)
    try:
        with pytest.raises(pg.PamcError):
            pg.pamc_dense_rows(hs)
    finally:
        pg.pamc_destroy(hs)


def test_dense_full_size_sweep_replay(pg):
    """The sweep at full size, n = 100,000 and R = 64 (the benchmark's
    instance and population), on sampled outputs the oracle computes one by
    one: from a seeded population set through the ABI, one step of one sweep
    at beta0; the first 1,024 positions of the order (four blocks, so the
    chains, the tiles and the tensor-core field update of earlier blocks all
    take part) are replayed sequentially on the CPU for every replica from
    their exact fields, with the oracle's draws, order and thresholds."""
    import torch
    n, R, seed, K = 100000, 64, 0, 1024
    params = dict(R=R, sweeps=1, steps=4, beta0=0.01, beta1=1.0, seed=11)
    wd = torch.empty((n, n), dtype=torch.int8, device="cuda")
    for r0 in range(0, n, 2000):
        wd[r0:r0 + 2000] = -W.dense_rows_torch(n, r0, min(n, r0 + 2000), seed, device="cuda")
    h = pg.pamc_create_dense(n, wd)
    del wd
    torch.cuda.empty_cache()
    try:
        pg.pamc_init(h, **params)
        rng = np.random.default_rng(7)
        S0 = np.where(rng.random((R, n)) < 0.5, 1, -1).astype(np.int8)
        pg.pamc_set_population(h, S0)
        pg.pamc_step(h, 1)
        S1, _, _, _ = pg.pamc_state(h, R, n)
    finally:
        pg.pamc_destroy(h)
    order = oracle.permutation(n, params["seed"], 0, 0)
    P = order[:K]
    JP = W.dense_rows_np(n, P, seed)                                   # couplings of the K rows
    hcur = (JP.astype(np.float32) @ S0.T.astype(np.float32)).round().astype(np.int64)   # exact: |h| < 2^24
    JPP = JP[:, P].astype(np.int64)                                    # couplings among the K positions
    key = (params["seed"] & 0xFFFFFFFF, params["seed"] >> 32)
    thr = {}
    s = S0[:, P].astype(np.int64).T.copy()                             # K x R
    for i in range(K):
        k = int(P[i])
        for g in range(R // 4):
            u = oracle.philox4x32_10((k, 0, 0, (oracle.TAG_FLIP << 24) | g), key)
            for q in range(4):
                r = 4 * g + q
                hv = int(hcur[i, r])
                if hv not in thr:
                    thr[hv] = oracle.thr_heatbath(params["beta0"], hv)
                new = 1 if int(u[q]) < thr[hv] else -1
                if new != s[i, r]:
                    hcur[i + 1:, r] += 2 * new * JPP[i + 1:, i]
                    s[i, r] = new
    np.testing.assert_array_equal(S1[:, P], s.T.astype(np.int8))
    assert (s.T != S0[:, P]).mean() > 0.2          # a hot step: the update path is exercised


def test_set_population_sparse_and_ranges(pg):
    inst = W.torus(12, 12, signed=True, seed=3)
    h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
    try:
        pg.pamc_init(h, R=6, steps=3, seed=2)
        S = np.ones((6, inst.n), dtype=np.int8)
        S[3, ::2] = -1
        pg.pamc_set_population(h, S)
        _, E, _, _ = pg.pamc_state(h, 6, inst.n)
        J = -inst.w.astype(np.int32)
        for r in range(6):
            assert E[r] == oracle.energy_ising(inst.row_ptr, inst.col, J, S[r])
        S[0, 0] = 0
        with pytest.raises(pg.PamcError):
            pg.pamc_set_population(h, S)
        with pytest.raises(pg.PamcError):
            pg.pamc_fields(h, 6, inst.n)
    finally:
        pg.pamc_destroy(h)
