"""Failure paths, made on purpose without faulting or hanging the GPU.

* A bounded device wait that runs out: the rounds of the cluster move's
  parallel greedy MIS are bounded (n + 1 always suffice); a host-set smaller
  bound makes a trial give up, which sets PAMC_ERR_TIMEOUT in the device
  status word.  pamc_sync reports it, no kernel is left waiting, and the
  context stays usable (a fresh run afterwards matches the oracle).
* Device allocation failure: an allocator that returns NULL from its k-th
  call on (for every k through pamc_create_csr and pamc_init) makes the call
  return PAMC_ERR_OOM, frees what it had taken, and leaves the handle usable
  for a later pamc_init.  Run in a fresh process, since the allocator is a
  process-wide setting made before any handle exists.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NCM_RUN = dict(R=32, sweeps=2, steps=150, beta0=0.5, beta1=6.0, stagnation=1, z_rst=120, cooldown_tau=5, seed=3)


@pytest.fixture(scope="module")
def pg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_25203_gb300 as pg
    pg.load()
    return pg


def test_mis_round_bound_running_out_reports_timeout(pg, monkeypatch):
    inst = W.torus(16, 16, signed=True, seed=2)
    monkeypatch.setenv("PAMC_NCM_MAX_ROUNDS", "0")
    s = pg.Solver(inst.row_ptr, inst.col, inst.w)
    s.init(**NCM_RUN)
    status = None
    for _ in range(NCM_RUN["steps"]):
        s.step(1)
        try:
            s.sync()
        except pg.PamcError as e:
            status = e.status
            break
    assert status == 7, "the bounded MIS rounds never ran out"
    s.close()
    # the context is intact: the same run without the bound matches the oracle
    monkeypatch.delenv("PAMC_NCM_MAX_ROUNDS")
    ref = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **NCM_RUN)
    s = pg.Solver(inst.row_ptr, inst.col, inst.w)
    s.init(**NCM_RUN)
    s.step(NCM_RUN["steps"])
    s.sync()
    ref.step(NCM_RUN["steps"])
    spins, E, _, _ = s.state()
    np.testing.assert_array_equal(spins, ref.spins())
    np.testing.assert_array_equal(E, ref.energy())
    assert ref.ctl()["ncm_flipped"] > 0
    s.close()


ALLOC_SCRIPT = r'''
import sys
sys.path.insert(0, ROOT)
import numpy as np
import torch
import oracle
import paper_2606_25203_gb300 as pg
import workloads as W

L = pg.load(torch_allocator=False)
state = {"left": 1 << 30, "live": 0}

def _alloc(nbytes, device, stream, ctx):
    if state["left"] <= 0:
        return None
    state["left"] -= 1
    state["live"] += 1
    return int(torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or 0))

def _free(ptr, device, stream, ctx):
    state["live"] -= 1
    torch.cuda.caching_allocator_delete(int(ptr))

cbs = (pg._ALLOC_FN(_alloc), pg._FREE_FN(_free))
assert L.pamc_set_allocator(cbs[0], cbs[1], None) == 0
inst = W.torus(12, 12, signed=True, seed=4)
params = dict(R=16, sweeps=2, steps=8, beta0=0.3, beta1=3.0, stagnation=1, z_rst=5, seed=2)

# creation: every allocation of the instance in turn fails
for k in range(2):
    state["left"] = k
    try:
        pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
        raise SystemExit("create succeeded with a failing allocator")
    except pg.PamcError as e:
        assert e.status == 5, e
    assert state["live"] == 0, state
state["left"] = 2
h = pg.pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w)
# initialisation: every allocation of the population in turn fails, then all succeed
fails = 0
for k in range(200):
    state["left"] = k
    try:
        pg.pamc_init(h, **params)
        break
    except pg.PamcError as e:
        assert e.status == 5, e
        assert state["live"] == 2, state          # only the instance stays allocated
        fails += 1
assert fails >= 10, fails
state["left"] = 1 << 30
pg.pamc_init(h, **params)
pg.pamc_step(h, params["steps"])
pg.pamc_sync(h)
ref = oracle.OracleRun(inst.row_ptr, inst.col, inst.w, **params)
ref.step(params["steps"])
spins, E, _, _ = pg.pamc_state(h, params["R"], inst.n)
assert np.array_equal(spins, ref.spins()) and np.array_equal(E, ref.energy())
pg.pamc_destroy(h)
assert state["live"] == 0, state
# a dense instance whose matrix cannot be allocated
state["left"] = 0
try:
    pg.pamc_create_dense(64, np.zeros((64, 64), dtype=np.int8))
    raise SystemExit("dense create succeeded with a failing allocator")
except pg.PamcError as e:
    assert e.status == 5, e
print("alloc-ok", fails)
'''


def test_allocation_failure_reports_oom(pg):
    script = ALLOC_SCRIPT.replace("ROOT", repr(ROOT))
    r = subprocess.run([sys.executable, "-c", script], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "alloc-ok" in r.stdout, r.stdout[-2000:] + r.stderr[-3000:]
