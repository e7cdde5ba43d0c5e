"""Diagnostics through the C ABI against the oracle's definitions: the
corrected pairwise Hamming histogram of the population (exact integers) and
the lineage of every slot through the resampling parent maps."""
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


@pytest.mark.parametrize("path", ["tensor", "cuda"])
@pytest.mark.parametrize("n,R,steps", [(300, 64, 6), (31, 33, 3), (1000, 70, 4), (40, 1, 2), (97, 5, 0),
                                       (2000, 300, 2)])
def test_hamming_matches_definition(pg, monkeypatch, path, n, R, steps):
    """Both paths: overlaps on the tensor cores (ragged n and R: padded K and
    rows, several 256 x 64 blocks) and XOR-popcount on the CUDA cores."""
    if path == "cuda":
        monkeypatch.setenv("PAMC_HAMMING", "cuda")
    inst = W.erdos_renyi(n, min(0.5, 8.0 / n), signed=True, seed=n)
    p = dict(R=R, sweeps=2, steps=max(steps, 1), seed=3, beta0=0.2, beta1=2.0)
    ref = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **p)
    h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
    try:
        pg.pamc_init(h, **p)
        pg.pamc_step(h, steps)
        ref.step(steps)
        spins, _, _, _ = pg.pamc_state(h, R, inst.n)
        np.testing.assert_array_equal(spins, ref.spins())
        hist, total = pg.pamc_hamming(h, inst.n)
        rh, rt = oracle.hamming_counts(ref.spins())
        np.testing.assert_array_equal(hist, rh)
        assert total == rt
        assert hist.sum() == R * (R - 1) // 2
    finally:
        pg.pamc_destroy(h)
        ref.close()


def test_hamming_large_population_exact(pg):
    """R=4096 on the 141x141 torus (8.4M pairs): the histogram equals the one
    from the overlap matrix q = S S^T (d = (n - q) / 2), computed with a plain
    fp32 matrix product (exact: integer sums below 2^24, TF32 off)."""
    import torch
    inst = W.c2a_torus141()
    R, n = 4096, inst.n
    h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
    try:
        pg.pamc_init(h, R=R, sweeps=2, steps=50, seed=1)
        pg.pamc_step(h, 3)
        hist, total = pg.pamc_hamming(h, n)
        spins, _, _, _ = pg.pamc_state(h, R, n)
    finally:
        pg.pamc_destroy(h)
    assert hist.sum() == R * (R - 1) // 2
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        S = torch.from_numpy(spins).cuda().float()
        q = (S @ S.T).round().long()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    d = (n - q) // 2
    iu = torch.triu_indices(R, R, offset=1, device=d.device)
    dc = torch.minimum(d[iu[0], iu[1]], n - d[iu[0], iu[1]])
    ref = torch.bincount(dc, minlength=n // 2 + 1).cpu().numpy()
    np.testing.assert_array_equal(hist, ref)
    assert total == int(dc.sum().item())


def test_hamming_dense(pg):
    inst = W.dense_csr(70, seed=3)
    p = dict(R=24, sweeps=2, steps=4, seed=5, beta0=0.05, beta1=0.5)
    J = -W.dense_rows_np(70, np.arange(70), 3).astype(np.int8)
    h = pg.pamc_create_dense(70, np.ascontiguousarray(J))
    try:
        pg.pamc_init(h, **p)
        pg.pamc_step(h, 4)
        spins, _, _, _ = pg.pamc_state(h, p["R"], 70)
        hist, total = pg.pamc_hamming(h, 70)
        rh, rt = oracle.hamming_counts(spins)
        np.testing.assert_array_equal(hist, rh)
        assert total == rt
    finally:
        pg.pamc_destroy(h)


def test_hamming_refuses_potts(pg):
    inst = W.torus(6, 6, signed=False, seed=1)
    h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
    try:
        pg.pamc_init(h, R=8, steps=2, kind=1)
        with pytest.raises(pg.PamcError):
            pg.pamc_hamming(h, inst.n)
    finally:
        pg.pamc_destroy(h)


@pytest.mark.parametrize("restart_reinit", [0, 1])
def test_lineage_follows_parent_maps(pg, restart_reinit):
    inst = W.gnm(400, 1100, signed=True, seed=8)
    p = dict(R=96, sweeps=1, steps=30, seed=2, beta0=0.3, beta1=4.0, z_rst=11, restart_reinit=restart_reinit)
    ref = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **p)
    h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
    fam = np.arange(p["R"], dtype=np.int32)
    try:
        pg.pamc_init(h, **p)
        restarted = False
        for t in range(p["steps"]):
            pg.pamc_step(h, 1)
            ref.step(1)
            parents, _ = ref.parents()
            fam = oracle.lineage_step(fam, parents, reinitialised=restarted and bool(restart_reinit))
            restarted = (t + 1) % p["z_rst"] == 0
            got, k = pg.pamc_lineage(h, p["R"])
            np.testing.assert_array_equal(got, fam, err_msg=f"step {t}")
            assert k == len(set(fam.tolist()))
        assert k < p["R"]          # resampling removed families
    finally:
        pg.pamc_destroy(h)
        ref.close()


def test_lineage_in_batch_equals_alone(pg):
    inst = W.torus(20, 20, signed=True, seed=4)
    p = dict(R=48, sweeps=2, steps=12, seed=6, beta0=0.5, beta1=3.0)
    h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
    pg.pamc_run(h, **p)
    ref, kref = pg.pamc_lineage(h, p["R"])
    pg.pamc_destroy(h)
    b = pg.pamc_batch_create(0)
    h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
    try:
        pg.pamc_init(h, **p)
        pg.pamc_batch_add(b, h)
        pg.pamc_batch_step(b, p["steps"])
        pg.pamc_batch_sync(b)
        got, k = pg.pamc_lineage(h, p["R"])
        np.testing.assert_array_equal(got, ref)
        assert k == kref
    finally:
        pg.pamc_batch_destroy(b)
        pg.pamc_destroy(h)
