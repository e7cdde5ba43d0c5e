"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the tests, the benchmark, the CPU oracle and the CUDA
path.  It holds none of the method's arithmetic: it only builds Max-Cut
instances (symmetric CSR with integer weights, or a dense symmetric int8
coupling matrix) and parameter sets.  The recipes stand in for the G-set graphs
(Sec. II, Sec. III.E-F) and the fully connected 100k-spin instance (Sec. III.G)
the paper uses, which are not available here:

* ``erdos_renyi``  -- each pair i<j is an edge with probability p (G1-G10 are
  n=800, p=0.06 random graphs with unit weights).
* ``gnm``          -- m distinct uniformly random edges (the sparse G55-G64
  class, average degree about 5.7), weights +1 or +-1.
* ``torus``        -- 2-D toroidal grid with +-1 weights (the G48-G81 toroidal
  instances).
* ``dense_pm1``    -- fully connected, J_ij = +-1 from a stateless 32-bit hash of
  (seed, min(i,j), max(i,j)), so any row can be regenerated on the CPU (numpy)
  or on the device (torch) without storing 10 GB on the host.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

M32 = 0xFFFFFFFF


@dataclass
class Instance:
    """Max-Cut instance: symmetric CSR (row_ptr, col, w) with zero diagonal."""
    name: str
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def edges(self) -> int:
        return self.nnz // 2


def csr_from_edges(n: int, ei: np.ndarray, ej: np.ndarray, w: np.ndarray, name: str) -> Instance:
    """Symmetric CSR with rows sorted by column from an undirected edge list."""
    ei = np.asarray(ei, dtype=np.int64)
    ej = np.asarray(ej, dtype=np.int64)
    w = np.asarray(w, dtype=np.int64)
    src = np.concatenate([ei, ej])
    dst = np.concatenate([ej, ei])
    ww = np.concatenate([w, w])
    order = np.lexsort((dst, src))
    src, dst, ww = src[order], dst[order], ww[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, src + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return Instance(name, n, row_ptr.astype(np.int32), dst.astype(np.int32), ww.astype(np.int32))


def _weights(rng: np.random.Generator, m: int, signed: bool) -> np.ndarray:
    if not signed:
        return np.ones(m, dtype=np.int64)
    return np.where(rng.integers(0, 2, size=m) == 1, 1, -1).astype(np.int64)


def erdos_renyi(n: int, p: float, signed: bool = False, seed: int = 0) -> Instance:
    rng = np.random.default_rng([seed, 1, n])
    iu, ju = np.triu_indices(n, k=1)
    keep = rng.random(iu.shape[0]) < p
    ei, ej = iu[keep], ju[keep]
    return csr_from_edges(n, ei, ej, _weights(rng, ei.shape[0], signed),
                          f"er_n{n}_p{p}_{'pm1' if signed else 'unit'}_s{seed}")


def gnm(n: int, m: int, signed: bool = True, seed: int = 0) -> Instance:
    rng = np.random.default_rng([seed, 2, n, m])
    seen = set()
    ei, ej = [], []
    while len(ei) < m:
        a = rng.integers(0, n, size=2 * (m - len(ei)) + 16)
        b = rng.integers(0, n, size=a.shape[0])
        for x, y in zip(a.tolist(), b.tolist()):
            if x == y:
                continue
            i, j = (x, y) if x < y else (y, x)
            code = i * n + j
            if code in seen:
                continue
            seen.add(code)
            ei.append(i)
            ej.append(j)
            if len(ei) == m:
                break
    ei = np.array(ei, dtype=np.int64)
    ej = np.array(ej, dtype=np.int64)
    return csr_from_edges(n, ei, ej, _weights(rng, m, signed),
                          f"gnm_n{n}_m{m}_{'pm1' if signed else 'unit'}_s{seed}")


def torus(rows: int, cols: int, signed: bool = True, seed: int = 0) -> Instance:
    rng = np.random.default_rng([seed, 3, rows, cols])
    idx = np.arange(rows * cols).reshape(rows, cols)
    right = np.roll(idx, -1, axis=1)
    down = np.roll(idx, -1, axis=0)
    ei = np.concatenate([idx.ravel(), idx.ravel()])
    ej = np.concatenate([right.ravel(), down.ravel()])
    # drop self loops / duplicates that appear on degenerate 1- or 2-wide tori
    a, b = np.minimum(ei, ej), np.maximum(ei, ej)
    code = a * (rows * cols) + b
    _, first = np.unique(code, return_index=True)
    first = np.sort(first)
    a, b = a[first], b[first]
    keep = a != b
    a, b = a[keep], b[keep]
    return csr_from_edges(rows * cols, a, b, _weights(rng, a.shape[0], signed),
                          f"torus_{rows}x{cols}_{'pm1' if signed else 'unit'}_s{seed}")


# ------------------------------------------------------------ dense +-1 instance
def _fmix32_np(h: np.ndarray) -> np.ndarray:
    h = h & M32
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & M32
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & M32
    h ^= h >> 16
    return h


def dense_rows_np(n: int, rows: np.ndarray, seed: int = 0) -> np.ndarray:
    """Rows of the dense +-1 coupling matrix (int8, zero diagonal) on the CPU."""
    rows = np.asarray(rows, dtype=np.uint64).reshape(-1, 1)
    j = np.arange(n, dtype=np.uint64).reshape(1, -1)
    lo = np.minimum(rows, j)
    hi = np.maximum(rows, j)
    s0 = np.uint64(seed & M32)
    s1 = np.uint64((seed >> 32) & M32)
    a = _fmix32_np((lo * np.uint64(0x9E3779B1) + s0) & np.uint64(M32))
    b = _fmix32_np(((a ^ hi) * np.uint64(0x85EBCA6B) + s1) & np.uint64(M32))
    J = np.where((b >> np.uint64(31)) == 1, 1, -1).astype(np.int8)
    J[rows.ravel()[:, None] == j.ravel()[None, :]] = 0
    return J


def dense_rows_torch(n: int, r0: int, r1: int, seed: int = 0, device="cpu"):
    """Rows r0..r1-1 of the same matrix with torch integer ops (for the device)."""
    import torch
    rows = torch.arange(r0, r1, dtype=torch.int64, device=device).view(-1, 1)
    j = torch.arange(n, dtype=torch.int64, device=device).view(1, -1)
    lo = torch.minimum(rows, j)
    hi = torch.maximum(rows, j)

    def fmix(h):
        h = h & M32
        h = h ^ (h >> 16)
        h = (h * 0x85EBCA6B) & M32
        h = h ^ (h >> 13)
        h = (h * 0xC2B2AE35) & M32
        h = h ^ (h >> 16)
        return h

    a = fmix((lo * 0x9E3779B1 + (seed & M32)) & M32)
    b = fmix(((a ^ hi) * 0x85EBCA6B + ((seed >> 32) & M32)) & M32)
    J = torch.where((b >> 31) == 1, 1, -1).to(torch.int8)
    J[rows.expand(-1, n) == j.expand(r1 - r0, -1)] = 0
    return J


def dense_csr(n: int, seed: int = 0) -> Instance:
    """Small dense instances as CSR (Max-Cut weights w = -J) for the oracle."""
    J = dense_rows_np(n, np.arange(n), seed).astype(np.int64)
    iu, ju = np.triu_indices(n, k=1)
    return csr_from_edges(n, iu, ju, -J[iu, ju], f"dense_n{n}_s{seed}")


# ------------------------------------------------------------ named workloads
def c1_er800(seed: int = 0) -> Instance:
    """Erdos-Renyi N=800, p=0.06, unit weights."""
    return erdos_renyi(800, 0.06, signed=False, seed=seed)


def c2a_torus141(seed: int = 0) -> Instance:
    """141x141 torus, N=19,881, 39,762 edges, +-1 weights."""
    return torus(141, 141, signed=True, seed=seed)


def c2b_sparse7000(seed: int = 0) -> Instance:
    """Random sparse N=7,000, average degree 5.7 (19,950 edges), +-1 weights."""
    return gnm(7000, int(round(7000 * 5.7 / 2)), signed=True, seed=seed)


def c3_sparse2000(seed: int = 0) -> Instance:
    """Random sparse N=2,000, average degree 12 (12,000 edges), unit weights."""
    return gnm(2000, 12000, signed=False, seed=seed)


def er_avg_degree(n: int, avg_deg: float, signed: bool = False, seed: int = 0) -> Instance:
    """Erdos-Renyi G(n, m) with m = round(n * avg_deg / 2) distinct uniform edges,
    drawn vectorised (oversample pairs, keep the first m distinct ones in draw
    order), so that n = 20,000 takes milliseconds."""
    m = int(round(n * avg_deg / 2))
    m = min(m, n * (n - 1) // 2)
    rng = np.random.default_rng([seed, 4, n, m])
    codes = np.zeros(0, dtype=np.int64)
    while True:
        k = 2 * m + 64
        a = rng.integers(0, n, size=k)
        b = rng.integers(0, n, size=k)
        keep = a != b
        lo, hi = np.minimum(a[keep], b[keep]), np.maximum(a[keep], b[keep])
        codes = np.concatenate([codes, lo * n + hi])
        _, first = np.unique(codes, return_index=True)
        if first.shape[0] >= m:
            break
    sel = codes[np.sort(first)[:m]]
    ei, ej = sel // n, sel % n
    return csr_from_edges(n, ei, ej, _weights(rng, m, signed),
                          f"er_n{n}_d{avg_deg}_{'pm1' if signed else 'unit'}_s{seed}")


@dataclass
class Request:
    """One solve request of a serving stream: an instance, its arrival time (s)
    and the problem asked: 0 Max-Cut, 1 Max-3-Cut."""
    rid: int
    inst: Instance
    arrival: float
    kind: int = 0


def serving_stream(count: int, rate: float, seed: int = 0, n_lo: int = 800, n_hi: int = 20000,
                   er_degree: float = 20.0, max3cut_frac: float = 0.0) -> list:
    """Solve requests with Poisson arrivals (exponential gaps, mean 1/rate s),
    N uniform in [n_lo, n_hi], the graph type drawn from Erdos-Renyi with unit
    weights, Erdos-Renyi with +-1 weights and a +-1 torus (side round(sqrt(N)),
    so N becomes side^2).  Erdos-Renyi requests have average degree er_degree
    (the G22-G31 / G43-G47 density class).  A fraction max3cut_frac of the
    requests (drawn from a stream of its own, so the instances do not depend
    on it) asks for Max-3-Cut, the others for Max-Cut."""
    kinds3 = np.random.default_rng([seed, 6, count]).random(count) < max3cut_frac
    rng = np.random.default_rng([seed, 5, count])
    gaps = rng.exponential(1.0 / rate, size=count) if rate > 0 else np.zeros(count)
    arrivals = np.cumsum(gaps) - gaps[0]
    sizes = rng.integers(n_lo, n_hi + 1, size=count)
    kinds = rng.integers(0, 3, size=count)
    out = []
    for i in range(count):
        n = int(sizes[i])
        s = seed * 100003 + i
        if kinds[i] == 0:
            inst = er_avg_degree(n, er_degree, signed=False, seed=s)
        elif kinds[i] == 1:
            inst = er_avg_degree(n, er_degree, signed=True, seed=s)
        else:
            side = max(3, int(round(np.sqrt(n))))
            inst = torus(side, side, signed=True, seed=s)
        out.append(Request(i, inst, float(arrivals[i]), 1 if kinds3[i] else 0))
    return out
