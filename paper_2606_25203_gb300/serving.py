"""Continuous-batching request loop over the batch entry points of libpamc.

Requests (a CSR instance, the problem -- Max-Cut, or Max-3-Cut with the
cascaded three-state sampler -- and an arrival time; run parameters shared) are
admitted while their device footprint (``pamc_footprint``: the instance, the
two spin buffers, energies, parents, counts and the schedule ring) fits the
HBM budget and a slot is free.  Every admitted population stays resident on
the device across its temperature steps; all of them advance together through
``pamc_batch_step`` (one captured CUDA graph per membership, one launch per
kernel type and size class per step), so requests that arrive while others run
join the mix as soon as memory and a slot free up.  A member that completed its
steps is retired, its best cut read back and its memory released.

The loop itself only does bookkeeping on the host; every step of every solve
runs in the library's kernels.  ``serve_sequential`` is the plain path for
comparison: one instance at a time, each run with ``pamc_run`` on its own.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import (pamc_batch_active, pamc_batch_add, pamc_batch_create, pamc_batch_destroy,
               pamc_batch_graph_builds, pamc_batch_launch_count, pamc_batch_retire, pamc_batch_step,
               pamc_best, pamc_create_csr, pamc_destroy, pamc_footprint, pamc_init, pamc_launch_count,
               pamc_run)


def request_params(params: dict, req) -> dict:
    """The run parameters of one request: the shared ones and its problem kind
    (0 Max-Cut, 1 Max-3-Cut; requests without a kind are Max-Cut)."""
    return dict(params, kind=int(getattr(req, "kind", 0)))


@dataclass
class Result:
    rid: int
    n: int
    cut: int
    arrival: float      # seconds after the start of the stream
    admitted: float
    finished: float
    spins: np.ndarray | None = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class ServeStats:
    results: list = field(default_factory=list)
    makespan: float = 0.0
    launches: int = 0
    graph_builds: int = 0
    peak_active: int = 0
    peak_bytes: int = 0

    @property
    def solves_per_s(self) -> float:
        return len(self.results) / self.makespan if self.makespan > 0 else 0.0

    def latency_pct(self, q: float) -> float:
        lat = np.array([r.latency for r in self.results])
        return float(np.percentile(lat, q)) if lat.size else 0.0


class Server:
    """Admits requests by HBM footprint and advances all admitted solves together.

    device: CUDA device index.  hbm_budget: device bytes the resident
    populations may take (default: half of the free memory at construction).
    max_active: most solves resident at once.  steps_per_tick: batch steps
    enqueued between two looks at the arrival queue; at most two ticks are in
    flight, so the host never runs far ahead of the device.
    """

    def __init__(self, device: int = 0, hbm_budget: int | None = None, max_active: int = 256,
                 steps_per_tick: int = 2, keep_spins: bool = False):
        import torch
        self.device = device
        self.torch = torch
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(device)
            hbm_budget = free // 2
        self.hbm_budget = int(hbm_budget)
        self.max_active = int(max_active)
        self.steps_per_tick = max(1, int(steps_per_tick))
        self.keep_spins = keep_spins
        self.stream = torch.cuda.Stream(device)          # batch steps
        self.admit_stream = torch.cuda.Stream(device)    # instance upload and initialisation
        self.batch = pamc_batch_create(device, self.stream.cuda_stream)

    def autotune(self, samples, params: dict, **kw) -> dict:
        """Pick the batched sweep's launch shape per size class on copies of
        ``samples`` (see ``tune.tune_batch_shapes``)."""
        from .tune import tune_batch_shapes
        return tune_batch_shapes(self.batch, samples, params, device=self.device, **kw)

    def close(self):
        if self.batch is not None:
            pamc_batch_destroy(self.batch)
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def serve(self, requests, params: dict, clock=time.perf_counter) -> ServeStats:
        """Serve a stream of ``workloads.Request`` (arrival times in seconds from
        the start) with the same run parameters ``params`` for every request."""
        torch = self.torch
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        active = {}            # handle value -> (request, handle, footprint, admitted)
        used = 0
        stats = ServeStats()
        ticks = deque()        # events of the ticks in flight
        staged = None          # (request, handle, footprint): created, waiting for memory
        builds0 = pamc_batch_graph_builds(self.batch)
        launches0 = pamc_batch_launch_count(self.batch)
        t0 = clock()
        while pending or active or staged:
            now = clock() - t0
            # admission: arrived requests, in arrival order, while memory and slots allow
            while (staged or (pending and pending[0].arrival <= now)) and len(active) < self.max_active:
                if staged is None:
                    req = pending.popleft()
                    h = pamc_create_csr(req.inst.n, req.inst.row_ptr, req.inst.col, req.inst.w,
                                        self.device, self.admit_stream.cuda_stream)
                    staged = (req, h, pamc_footprint(h, **request_params(params, req)))
                req, h, fp = staged
                if active and used + fp > self.hbm_budget:
                    break          # wait for a retirement
                pamc_init(h, **request_params(params, req))
                pamc_batch_add(self.batch, h)
                active[h.value] = (req, h, fp, clock() - t0)
                used += fp
                staged = None
                stats.peak_active = max(stats.peak_active, len(active))
                stats.peak_bytes = max(stats.peak_bytes, used)
            if not active:
                if pending and staged is None:
                    wait = pending[0].arrival - (clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
                continue
            if pamc_batch_active(self.batch) > 0:
                pamc_batch_step(self.batch, self.steps_per_tick)
                ev = torch.cuda.Event()
                ev.record(self.stream)
                ticks.append(ev)
                if len(ticks) > 2:
                    ticks.popleft().synchronize()
            done = pamc_batch_retire(self.batch)
            if done:
                ticks.clear()      # retire waited for the batch stream
                fin = clock() - t0
                for h in done:
                    req, hh, fp, adm = active.pop(h.value)
                    cut, spins = pamc_best(hh, req.inst.n)
                    stats.results.append(Result(req.rid, req.inst.n, int(cut), req.arrival, adm, fin,
                                                spins if self.keep_spins else None))
                    pamc_destroy(hh)
                    used -= fp
        stats.makespan = clock() - t0
        stats.graph_builds = pamc_batch_graph_builds(self.batch) - builds0
        stats.launches = pamc_batch_launch_count(self.batch) - launches0
        return stats


def serve_sequential(requests, params: dict, device: int = 0, keep_spins: bool = False,
                     clock=time.perf_counter) -> ServeStats:
    """The plain path: requests in arrival order, one ``pamc_run`` at a time
    (each kernel launched for one instance), on one stream."""
    import torch
    stream = torch.cuda.Stream(device)
    stats = ServeStats()
    t0 = clock()
    for req in sorted(requests, key=lambda r: r.arrival):
        wait = req.arrival - (clock() - t0)
        if wait > 0:
            time.sleep(wait)
        adm = clock() - t0
        h = pamc_create_csr(req.inst.n, req.inst.row_ptr, req.inst.col, req.inst.w, device,
                            stream.cuda_stream)
        try:
            pamc_run(h, **request_params(params, req))
            cut, spins = pamc_best(h, req.inst.n)
            stats.launches += pamc_launch_count(h)
        finally:
            pamc_destroy(h)
        stats.results.append(Result(req.rid, req.inst.n, int(cut), req.arrival, adm, clock() - t0,
                                    spins if keep_spins else None))
    stats.makespan = clock() - t0
    return stats
