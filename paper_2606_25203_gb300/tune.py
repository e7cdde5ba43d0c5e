"""Autotuner for the batched sweep's launch shape per size class.

For every size class (``pamc_size_class``: n <= 2048, <= 8192, larger) that the
sample instances cover, the samples of that class are loaded into a throwaway
batch and each candidate shape -- replica groups (of four replicas) per CTA,
warps per group, lanes per vertex, and where the groups' spin words live
(shared memory, or device memory with no shared-memory limit on groups per
SM) -- is timed with CUDA events over a few batch steps; the fastest one is
set on the caller's batch.  A shape changes speed only, never results, so
tuning on copies of representative instances is safe.
"""
from __future__ import annotations

from . import (pamc_batch_add, pamc_batch_create, pamc_batch_destroy, pamc_batch_set_lanes,
               pamc_batch_set_placement, pamc_batch_set_shape, pamc_batch_step, pamc_create_csr, pamc_destroy,
               pamc_init, pamc_size_class)

# (groups per CTA, warps per group, lanes per vertex, spin words in device
# memory); several lanes per vertex only pay off with wide groups, and device
# memory only with one lane per vertex
CANDIDATES = (tuple((g, w, 1, 0) for g in (1, 2, 4, 8) for w in (1, 2, 4, 8, 16) if g * w <= 32) +
              tuple((g, w, l, 0) for g in (1, 2) for w in (4, 8, 16, 32) for l in (2, 4) if g * w <= 32) +
              tuple((g, w, 1, 1) for g in (1, 2, 4) for w in (4, 8, 16) if g * w <= 32))


def tune_batch_shapes(batch, samples, params: dict, steps: int = 3, rounds: int = 2, device: int = 0,
                      candidates=CANDIDATES) -> dict:
    """samples: instances with ``n``, ``row_ptr``, ``col``, ``w`` (numpy CSR),
    or (instance, kind) pairs -- kind 0 Max-Cut, 1 Max-3-Cut -- so that a
    class's shape is timed on the mix of problems it will serve.
    params: run parameters of the served requests (R, sweeps, rule, ...).
    candidates: (groups, warps), (groups, warps, lanes) or (groups, warps,
    lanes, device-memory spin words) tuples.
    Returns {size_class: (groups_per_cta, warps_per_group, lanes_per_vertex,
    ms_per_step, device_memory_spins)}."""
    candidates = tuple(tuple(c) + (1, 0)[len(c) - 2:] if len(c) < 4 else tuple(c) for c in candidates)
    import torch
    by_class = {}
    for smp in samples:
        inst, kind = smp if isinstance(smp, tuple) else (smp, 0)
        by_class.setdefault(pamc_size_class(inst.n), []).append((inst, kind))
    p = dict(params)
    p["steps"] = 1 << 20          # the throwaway runs never finish
    p.pop("target_cut", None)
    stream = torch.cuda.Stream(device)
    chosen = {}
    for cls, insts in sorted(by_class.items()):
        hs = []
        tmp = pamc_batch_create(device, stream.cuda_stream)
        try:
            for inst, kind in insts:
                h = pamc_create_csr(inst.n, inst.row_ptr, inst.col, inst.w, device, stream.cuda_stream)
                hs.append(h)
                pamc_init(h, **dict(p, kind=kind))
                pamc_batch_add(tmp, h)
            best = {}
            for _ in range(rounds):          # candidates interleaved, best of the rounds
                for g, w, lv, gm in candidates:
                    pamc_batch_set_shape(tmp, cls, g, w)
                    pamc_batch_set_lanes(tmp, cls, lv)
                    pamc_batch_set_placement(tmp, cls, bool(gm))
                    pamc_batch_step(tmp, 1)  # capture and warm up
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    pamc_batch_step(tmp, steps)
                    b.record(stream)
                    b.synchronize()
                    ms = a.elapsed_time(b) / steps
                    best[(g, w, lv, gm)] = min(ms, best.get((g, w, lv, gm), float("inf")))
            (g, w, lv, gm), ms = min(best.items(), key=lambda kv: kv[1])
            pamc_batch_set_shape(batch, cls, g, w)
            pamc_batch_set_lanes(batch, cls, lv)
            pamc_batch_set_placement(batch, cls, bool(gm))
            chosen[cls] = (g, w, lv, ms, gm)
        finally:
            pamc_batch_destroy(tmp)
            for h in hs:
                pamc_destroy(h)
    return chosen
