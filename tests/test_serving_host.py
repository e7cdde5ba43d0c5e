"""Host logic of the continuous-batching server, on CPU: the library's batch
entry points are replaced by a small model of a batch (members advance one
temperature step per batch step and finish after ``steps``), so admission by
footprint, the slot limit, retirement and the bookkeeping of every request
can be checked without a GPU.  The device path itself is covered by
``test_gpu_batch.py`` (every member identical to its run alone)."""
import ctypes
import os
import sys
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from paper_2606_25203_gb300 import serving  # noqa: E402


class FakeLib:
    """A batch as the library keeps it: members with a step counter."""

    def __init__(self, bytes_per_vertex=1000):
        self.bpv = bytes_per_vertex
        self.next = 0x1000
        self.n = {}          # handle -> n
        self.steps = {}      # handle -> steps of its run
        self.done = {}       # handle -> steps done
        self.members = []
        self.resident = set()
        self.max_resident = 0
        self.log = []        # ("add", n) / ("retire", n) in order

    def create(self, n, rp, col, w, device, stream):
        h = ctypes.c_void_p(self.next)
        self.next += 16
        self.n[h.value] = n
        self.resident.add(h.value)
        return h

    def footprint(self, h, **p):
        return self.n[h.value] * self.bpv

    def init(self, h, **p):
        self.steps[h.value] = p["steps"]
        self.done[h.value] = 0

    def add(self, b, h):
        self.members.append(h.value)
        self.max_resident = max(self.max_resident, len(self.members))
        self.log.append(("add", self.n[h.value]))

    def active(self, b):
        return sum(1 for m in self.members if self.done[m] < self.steps[m])

    def step(self, b, k):
        for m in self.members:
            self.done[m] = min(self.steps[m], self.done[m] + k)

    def retire(self, b, max_out=4096):
        fin = [m for m in self.members if self.done[m] >= self.steps[m]][:max_out]
        for m in fin:
            self.members.remove(m)
            self.log.append(("retire", self.n[m]))
        return [ctypes.c_void_p(m) for m in fin]

    def best(self, h, n):
        assert self.n[h.value] == n
        return 1000 + n, np.zeros(n, dtype=np.int8)

    def destroy(self, h):
        assert h.value not in self.members
        self.resident.discard(h.value)


class FakeClock:
    def __init__(self, tick=0.001):
        self.t = 0.0
        self.tick = tick

    def __call__(self):
        self.t += self.tick
        return self.t


def make_server(monkeypatch, lib, budget, max_active, steps_per_tick=1):
    for name, fn in (("pamc_create_csr", lib.create), ("pamc_footprint", lib.footprint),
                     ("pamc_init", lib.init), ("pamc_batch_add", lib.add),
                     ("pamc_batch_active", lib.active), ("pamc_batch_step", lib.step),
                     ("pamc_batch_retire", lib.retire), ("pamc_best", lib.best),
                     ("pamc_destroy", lib.destroy),
                     ("pamc_batch_graph_builds", lambda b: 0), ("pamc_batch_launch_count", lambda b: 0)):
        monkeypatch.setattr(serving, name, fn)

    class Event:
        def record(self, stream):
            pass

        def synchronize(self):
            pass

    s = serving.Server.__new__(serving.Server)
    s.device = 0
    s.torch = types.SimpleNamespace(cuda=types.SimpleNamespace(Event=Event))
    s.hbm_budget = budget
    s.max_active = max_active
    s.steps_per_tick = steps_per_tick
    s.keep_spins = False
    s.stream = s.admit_stream = types.SimpleNamespace(cuda_stream=None)
    s.batch = object()
    return s


def requests(sizes, arrivals=None):
    """Requests whose instances carry only n (the fake library never reads the CSR)."""
    return [W.Request(rid=i, inst=types.SimpleNamespace(n=n, row_ptr=None, col=None, w=None),
                      arrival=0.0 if arrivals is None else arrivals[i])
            for i, n in enumerate(sizes)]


def test_every_request_served_once_with_its_own_result(monkeypatch):
    lib = FakeLib()
    srv = make_server(monkeypatch, lib, budget=10**12, max_active=64)
    reqs = requests([800, 1200, 3000, 20000, 950])
    st = srv.serve(reqs, dict(steps=7), clock=FakeClock())
    assert sorted(r.rid for r in st.results) == list(range(5))
    for r in st.results:
        assert r.cut == 1000 + r.n
        assert r.arrival <= r.admitted <= r.finished
    assert not lib.members and not lib.resident      # every handle retired and destroyed
    assert st.peak_active == 5                        # all resident together: one batch


def test_admission_respects_the_footprint_budget_and_arrival_order(monkeypatch):
    lib = FakeLib(bytes_per_vertex=1000)
    # budget for 2,500 vertices: at most two of these requests resident at once
    srv = make_server(monkeypatch, lib, budget=2_500_000, max_active=64)
    sizes = [1000, 1200, 900, 1100, 800, 1000]
    st = srv.serve(requests(sizes), dict(steps=5), clock=FakeClock())
    assert len(st.results) == len(sizes)
    assert st.peak_bytes <= 2_500_000 and st.peak_active == 2
    adds = [n for op, n in lib.log if op == "add"]
    assert adds == sizes                              # admitted in arrival order
    # replay the log: the resident footprint never exceeds the budget
    used = 0
    for op, n in lib.log:
        used += n * 1000 if op == "add" else -n * 1000
        assert used <= 2_500_000


def test_a_request_larger_than_the_budget_runs_alone(monkeypatch):
    lib = FakeLib(bytes_per_vertex=1000)
    srv = make_server(monkeypatch, lib, budget=1_500_000, max_active=64)
    st = srv.serve(requests([1000, 5000, 1000]), dict(steps=3), clock=FakeClock())
    assert len(st.results) == 3
    resident = 0
    for op, n in lib.log:
        resident += 1 if op == "add" else -1
        if op == "add" and n == 5000:
            assert resident == 1                      # admitted only into an empty batch


def test_slot_limit_and_joining_while_others_run(monkeypatch):
    lib = FakeLib()
    srv = make_server(monkeypatch, lib, budget=10**12, max_active=4, steps_per_tick=2)
    # three requests start together; four more arrive while they are stepping:
    # one joins the running batch at once, the others wait for free slots
    arrivals = [0.0, 0.0, 0.0, 0.004, 0.004, 0.004, 0.004]
    st = srv.serve(requests([800] * 7, arrivals), dict(steps=40), clock=FakeClock(0.001))
    assert len(st.results) == 7 and st.peak_active == 4 and lib.max_resident == 4
    first_retire = next(i for i, (op, _) in enumerate(lib.log) if op == "retire")
    assert sum(1 for op, _ in lib.log[:first_retire] if op == "add") == 4
    joined = sorted(st.results, key=lambda r: r.rid)[3]
    assert 0.004 <= joined.admitted < min(r.finished for r in st.results)
    for r in st.results:
        assert r.admitted >= r.arrival


def test_latency_percentiles_and_throughput():
    st = serving.ServeStats()
    for i, lat in enumerate([1.0, 2.0, 3.0, 4.0]):
        st.results.append(serving.Result(i, 10, 0, 0.0, 0.0, lat))
    st.makespan = 4.0
    assert st.solves_per_s == pytest.approx(1.0)
    assert st.latency_pct(50) == pytest.approx(2.5)
    assert st.latency_pct(100) == pytest.approx(4.0)
