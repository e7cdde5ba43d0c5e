"""One population split over several processes, one GPU each.

The population step of Algorithm 1 (Eq. 1-2) is global over the R replicas:
slot m of the next population copies old replica parent[m], wherever that
replica lives.  Each process holds an equal block of slots (R a multiple of
4 x processes) and an iteration exchanges twice:

1. all-gather of the R energies (int64) -- every process then runs the same
   reweighting, integer prefix scan and controller on them and obtains the
   same parent map, NCM targets and decisions;
2. all-to-all of the parent replicas whose slot lives on another process
   (n int8 each; the plan is computed by every process from the parent map,
   so no sizes are exchanged).  Systematic resampling gives a nondecreasing
   parent map, so only replicas near the block edges move.

After the sweeps the energies are gathered again for M* and the controller,
and that gather also serves the next iteration unless a restart re-draws the
population.  The random draws are keyed by each replica's index in the whole
population, so the split run equals the single-process run bit for bit.

``run_step`` is the exchange of one iteration over any shard (the library's
``LibShard`` below; tests also drive it with CPU shards) and any
communicator with ``all_gather``, ``all_to_all`` and ``broadcast``
(``TorchComm``: ``torch.distributed``, NCCL for CUDA tensors).
"""
from __future__ import annotations

import numpy as np

from . import (load, pamc_create_csr, pamc_create_dense, pamc_destroy, pamc_shard_best, pamc_shard_control,
               pamc_shard_energies,
               pamc_shard_init, pamc_shard_pack, pamc_shard_plan, pamc_shard_range, pamc_shard_resample,
               pamc_shard_sweep)


class TorchComm:
    """The collectives of ``run_step`` on a torch.distributed group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def all_gather(self, out, inp):
        self.dist.all_gather_into_tensor(out, inp, group=self.group)

    def all_to_all(self, recv, send, recv_splits, send_splits):
        self.dist.all_to_all_single(recv, send, output_split_sizes=list(recv_splits),
                                    input_split_sizes=list(send_splits), group=self.group)

    def broadcast(self, t, src: int):
        """src: the rank within the group."""
        g = src if self.group is None else self.dist.get_global_rank(self.group, src)
        self.dist.broadcast(t, g, group=self.group)


def run_step(shard, comm) -> None:
    """One iteration of Algorithm 1 for this process's share of the population.

    shard provides R, n, rank, nranks, count, the buffers E_own (count int64)
    and E_all (R int64), the flags e_all_valid and redraws, rows(k) (a
    buffer of k * n int8 on its device) and the five calls energies,
    resample, pack, sweep and control (the pamc_shard_* calls of
    include/pamc.h)."""
    if not shard.e_all_valid:
        shard.energies(shard.E_own)
        comm.all_gather(shard.E_all, shard.E_own)
    parent = shard.resample(shard.E_all)
    send_counts, send_rows, recv_counts, local_parent = pamc_shard_plan(shard.R, shard.nranks, shard.rank, parent)
    n_send, n_recv = int(send_counts.sum()), int(recv_counts.sum())
    send = shard.rows(n_send)
    shard.pack(send_rows, send)
    recv = shard.rows(n_recv)
    comm.all_to_all(recv, send, (recv_counts.astype(np.int64) * shard.n).tolist(),
                    (send_counts.astype(np.int64) * shard.n).tolist())
    shard.sweep(shard.E_all, local_parent, recv, n_recv, shard.E_own)
    comm.all_gather(shard.E_all, shard.E_own)
    shard.control(shard.E_all, shard.E_own)
    shard.e_all_valid = not shard.redraws
    shard.moved += n_recv


def best(shard, comm):
    """(M*, its configuration) on every process: the process holding it
    broadcasts the spins."""
    import torch
    cut, spins, owned = shard.best()
    flags = torch.zeros(comm.size, dtype=torch.int64, device=shard.E_all.device)
    mine = torch.tensor([1 if owned else 0], dtype=torch.int64, device=shard.E_all.device)
    comm.all_gather(flags, mine)
    owners = torch.nonzero(flags.cpu()).reshape(-1).tolist()
    if not owners:
        return cut, None
    buf = shard.rows(1)
    if owned:
        buf.copy_(torch.as_tensor(spins, dtype=torch.int8).to(buf.device))
    comm.broadcast(buf, owners[0])
    return cut, buf.cpu().numpy().copy()


class LibShard:
    """This process's share of a population, on the library (one GPU).

    The handle runs on the current torch stream of its device, so the
    collectives torch issues afterwards are ordered behind its kernels."""

    def __init__(self, row_ptr, col, w, rank: int, nranks: int, device: int = 0, dense_w=None, **params):
        """A CSR instance (row_ptr, col, w), or a dense one (dense_w: n x n
        int8 weights, host array or CUDA tensor; row_ptr, col, w None)."""
        import torch
        load()
        self.torch = torch
        self.dev = torch.device("cuda", device)
        if dense_w is not None:
            self.n = int(dense_w.shape[0])
            self.h = pamc_create_dense(self.n, dense_w, device=device)
        else:
            rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
            self.n = len(rp) - 1
            self.h = pamc_create_csr(self.n, rp, col, w, device=device)
        self.p = pamc_shard_init(self.h, rank, nranks, **params)
        self.R, self.rank, self.nranks = int(self.p.R), int(rank), int(nranks)
        self.base, self.count = pamc_shard_range(self.R, nranks, rank)
        self.redraws = self.p.z_rst > 0 and self.p.restart_reinit != 0
        self.E_own = torch.empty(self.count, dtype=torch.int64, device=self.dev)
        self.E_all = torch.empty(self.R, dtype=torch.int64, device=self.dev)
        self.e_all_valid = False
        self.moved = 0   # replicas received so far

    def rows(self, k: int):
        return self.torch.empty(int(k) * self.n, dtype=self.torch.int8, device=self.dev)

    def energies(self, E_own):
        pamc_shard_energies(self.h, E_own)

    def resample(self, E_all):
        return pamc_shard_resample(self.h, E_all)

    def pack(self, rows, send):
        pamc_shard_pack(self.h, rows, send)

    def sweep(self, E_all, local_parent, recv, nimports, E_own):
        pamc_shard_sweep(self.h, E_all, local_parent, recv, nimports, E_own)

    def control(self, E_all, E_own):
        pamc_shard_control(self.h, E_all, E_own)

    def best(self):
        return pamc_shard_best(self.h)

    def close(self):
        if self.h is not None:
            pamc_destroy(self.h)
            self.h = None


class ShardedSolver:
    """One population of R replicas split over the processes of a
    torch.distributed group (NCCL, one GPU per process): every process
    constructs it with the same instance and parameters."""

    def __init__(self, row_ptr, col, w, device: int = 0, group=None, **params):
        self.comm = TorchComm(group)
        self.shard = LibShard(row_ptr, col, w, self.comm.rank, self.comm.size, device=device, **params)

    def step(self, nsteps: int = 1):
        for _ in range(int(nsteps)):
            run_step(self.shard, self.comm)

    def best(self):
        return best(self.shard, self.comm)

    def close(self):
        self.shard.close()
