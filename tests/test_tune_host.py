"""Host logic of the launch-shape autotuner, on CPU: the library's batch
calls and CUDA events are replaced by a cost model, and the tuner must set,
per size class, the shape the model times fastest (best over its rounds), on
the caller's batch only, and release every throwaway handle."""
import ctypes
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
from paper_2606_25203_gb300 import tune  # noqa: E402


class Model:
    """Batches whose step time depends on the shape set for the class."""

    def __init__(self, cost):
        self.cost = cost              # (cls, g, w, lv, round) -> ms
        self.shape = {}               # (batch, cls) -> (g, w)
        self.lanes = {}               # (batch, cls) -> lv
        self.place = {}               # (batch, cls) -> spin words in device memory
        self.members = {}             # batch -> [classes]
        self.created, self.destroyed = [], []
        self.batches = []
        self.calls = 0
        self.next = 0x100

    def size_class(self, n):
        return 0 if n <= 2048 else (1 if n <= 8192 else 2)

    def batch_create(self, device, stream):
        b = object()
        self.batches.append(b)
        self.members[b] = []
        return b

    def create(self, n, *a):
        h = ctypes.c_void_p(self.next)
        self.next += 8
        self.created.append((h.value, n))
        return h

    def init(self, h, **p):
        assert p["steps"] >= 1 << 20 and "target_cut" not in p
        self.kinds = getattr(self, "kinds", []) + [(dict(self.created)[h.value], p.get("kind", 0))]

    def add(self, b, h):
        n = dict(self.created)[h.value]
        self.members[b].append(self.size_class(n))

    def set_shape(self, b, cls, g, w):
        self.shape[(b, cls)] = (g, w)

    def set_lanes(self, b, cls, lv):
        self.lanes[(b, cls)] = lv

    def set_placement(self, b, cls, gm):
        self.place[(b, cls)] = bool(gm)

    def step(self, b, k):
        self.last = (b, k)

    def batch_destroy(self, b):
        pass

    def destroy(self, h):
        self.destroyed.append(h.value)


def test_tuner_sets_the_fastest_shape_per_class(monkeypatch):
    # class 0 is fastest at (2, 4, 2) with spin words on chip; class 2 at
    # (1, 16, 1) with spin words in device memory; the second timing pass adds noise
    def cost(cls, g, w, lv, gm, rnd):
        best = {0: (2, 4, 2, 0), 2: (1, 16, 1, 1)}[cls]
        d = abs(g - best[0]) + abs(w - best[1]) / 4 + abs(lv - best[2]) + 0.3 * abs(gm - best[3])
        return 1.0 + d + (0.5 if rnd == 1 else 0.0)

    m = Model(cost)
    state = {"round": 0, "count": 0}
    ncand = len(tune.CANDIDATES)

    class Event:
        def __init__(self, enable_timing=False):
            pass

        def record(self, stream):
            self.when = m.last

        def synchronize(self):
            pass

        def elapsed_time(self, other):
            b, _ = m.last
            cls = next(c for (bb, c) in m.shape if bb is b)
            g, w = m.shape[(b, cls)]
            lv = m.lanes[(b, cls)]
            gm = int(m.place[(b, cls)])
            rnd = state["count"] // ncand
            state["count"] += 1
            return cost(cls, g, w, lv, gm, rnd % 2) * 3

    monkeypatch.setattr(torch.cuda, "Stream", lambda device=0: types.SimpleNamespace(cuda_stream=None))
    monkeypatch.setattr(torch.cuda, "Event", Event)
    for name, fn in (("pamc_size_class", m.size_class), ("pamc_batch_create", m.batch_create),
                     ("pamc_create_csr", m.create), ("pamc_init", m.init), ("pamc_batch_add", m.add),
                     ("pamc_batch_set_shape", m.set_shape), ("pamc_batch_set_lanes", m.set_lanes),
                     ("pamc_batch_set_placement", m.set_placement),
                     ("pamc_batch_step", m.step), ("pamc_batch_destroy", m.batch_destroy),
                     ("pamc_destroy", m.destroy)):
        monkeypatch.setattr(tune, name, fn)

    caller = object()
    samples = [types.SimpleNamespace(n=n, row_ptr=None, col=None, w=None) for n in (900, 1500, 12000)]
    samples[1] = (samples[1], 1)                    # a Max-3-Cut sample, given as (instance, kind)
    chosen = tune.tune_batch_shapes(caller, samples, dict(R=64, sweeps=2, steps=10, target_cut=5))
    assert set(chosen) == {0, 2}
    assert chosen[0][:3] == (2, 4, 2) and chosen[2][:3] == (1, 16, 1)
    assert chosen[0][3] == pytest.approx(1.0) and chosen[2][3] == pytest.approx(1.0)   # best round
    assert chosen[0][4] == 0 and chosen[2][4] == 1
    assert m.shape[(caller, 0)] == (2, 4) and m.lanes[(caller, 0)] == 2 and not m.place[(caller, 0)]
    assert m.shape[(caller, 2)] == (1, 16) and m.lanes[(caller, 2)] == 1 and m.place[(caller, 2)]
    assert (caller, 1) not in m.shape                       # no sample of class 1: untouched
    assert sorted(m.destroyed) == sorted(h for h, _ in m.created)
    assert sorted(m.kinds) == [(900, 0), (1500, 1), (12000, 0)]     # each sample run as its problem
