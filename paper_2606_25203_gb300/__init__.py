"""GB300 (sm_103a) augmented Population Annealing Monte Carlo.

Thin Python binding of the C ABI in ``include/pamc.h`` (libpamc.so): argument
marshalling only, every step of a run executes in the library's CUDA kernels.
The functions carry the C names (``pamc_create_csr``, ``pamc_init``,
``pamc_step``, ``pamc_run``, ``pamc_best``, ...).  PyTorch provides the device
memory (its caching allocator is registered with the library) and the stream.

There is no CPU fallback: importing the package without the built library or
a CUDA device raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "PamcError", "Params", "load", "pamc_create_csr", "pamc_create_dense", "pamc_init",
    "pamc_step", "pamc_sync", "pamc_run", "pamc_best", "pamc_state", "pamc_control_state",
    "pamc_launch_count", "pamc_sweep_shape", "pamc_dense_rows", "pamc_weight_sum", "pamc_last_error", "pamc_destroy", "Solver",
    "pamc_sweeps_noalloc", "pamc_footprint", "pamc_batch_create", "pamc_batch_add", "pamc_batch_step",
    "pamc_batch_retire", "pamc_batch_size", "pamc_batch_active", "pamc_batch_launch_count",
    "pamc_batch_graph_builds", "pamc_batch_sync", "pamc_batch_destroy", "pamc_size_class",
    "pamc_batch_set_shape", "pamc_batch_get_shape", "pamc_batch_set_lanes", "pamc_batch_get_lanes", "pamc_hamming", "pamc_lineage", "pamc_set_population", "pamc_fields",
    "pamc_control_history", "pamc_sweep_mode", "pamc_set_sweep_timing", "pamc_sweep_stats",
    "pamc_batch_set_placement", "pamc_batch_get_placement", "pamc_shard_range", "pamc_shard_init",
    "pamc_shard_energies", "pamc_shard_resample", "pamc_shard_plan", "pamc_shard_pack", "pamc_shard_sweep",
    "pamc_shard_control", "pamc_shard_best", "pamc_save", "pamc_load",
]

STATUS = {0: "PAMC_OK", 1: "PAMC_ERR_ARG", 2: "PAMC_ERR_ASYM", 3: "PAMC_ERR_DIAG",
          4: "PAMC_ERR_RANGE", 5: "PAMC_ERR_OOM", 6: "PAMC_ERR_CUDA", 7: "PAMC_ERR_TIMEOUT",
          8: "PAMC_ERR_STATE"}
STATUS_CODES = {v: k for k, v in STATUS.items()}


class PamcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    """Mirror of ``pamc_params``."""
    _fields_ = [
        ("kind", ctypes.c_int32), ("rule", ctypes.c_int32), ("R", ctypes.c_int32),
        ("sweeps", ctypes.c_int32), ("steps", ctypes.c_int32),
        ("beta0", ctypes.c_double), ("beta1", ctypes.c_double),
        ("stagnation", ctypes.c_int32), ("z_rst", ctypes.c_int32),
        ("cooldown_tau", ctypes.c_int32), ("n_top", ctypes.c_int32), ("mis_trials", ctypes.c_int32),
        ("win_short", ctypes.c_int32), ("win_long", ctypes.c_int32),
        ("max_distinct_short", ctypes.c_int32), ("max_distinct_long", ctypes.c_int32),
        ("reheat_factor", ctypes.c_double), ("target_cut", ctypes.c_int64),
        ("seed", ctypes.c_uint64), ("restart_reinit", ctypes.c_int32), ("resample", ctypes.c_int32),
        ("K", ctypes.c_int32), ("gamma", ctypes.c_double),
    ]


DEFAULTS = dict(kind=0, rule=0, R=16, sweeps=1, steps=10, beta0=0.1, beta1=3.0, stagnation=0,
                z_rst=0, cooldown_tau=10, n_top=0, mis_trials=4, win_short=25, win_long=40,
                max_distinct_short=3, max_distinct_long=5, reheat_factor=0.8, target_cut=-1,
                seed=0, restart_reinit=1, resample=1, K=3, gamma=1.0)

# limits of pamc_sweeps_noalloc (PAMC_NOALLOC_MAX_* in include/pamc.h)
NOALLOC_MAX_N, NOALLOC_MAX_NNZ, NOALLOC_MAX_SWEEPS, NOALLOC_MAX_R = 32768, 262144, 8, 16384

_lib = None
_alloc_cbs = None

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p,
                             ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)


def _register_torch_allocator(L):
    """Route the library's device allocations through torch's caching allocator."""
    global _alloc_cbs
    import torch

    def _alloc(nbytes, device, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or 0))
        except Exception:   # allocation failure is reported as NULL (PAMC_ERR_OOM)
            return None

    def _free(ptr, device, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    _alloc_cbs = (_ALLOC_FN(_alloc), _FREE_FN(_free))
    rc = L.pamc_set_allocator(_alloc_cbs[0], _alloc_cbs[1], None)
    if rc != 0:
        raise PamcError(rc, "pamc_set_allocator failed")


def load(build_if_missing: bool = True, torch_allocator: bool = True):
    """Load libpamc.so (building it with nvcc if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"libpamc.so is not built ({path}); run __graft_entry__.build()")
        path = _build.build()
    L = ctypes.CDLL(path)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.pamc_set_allocator.argtypes = [_ALLOC_FN, _FREE_FN, P]
    L.pamc_create_csr.argtypes = [i32, P, P, P, ctypes.c_int, P, ctypes.POINTER(P)]
    L.pamc_create_dense.argtypes = [i32, P, ctypes.c_int, ctypes.c_int, P, ctypes.POINTER(P)]
    L.pamc_init.argtypes = [P, ctypes.POINTER(Params)]
    L.pamc_step.argtypes = [P, i32]
    L.pamc_sync.argtypes = [P]
    L.pamc_run.argtypes = [P, ctypes.POINTER(Params)]
    L.pamc_best.argtypes = [P, P, P]
    L.pamc_state.argtypes = [P, P, P, P, P]
    L.pamc_control_state.argtypes = [P, P, P]
    L.pamc_launch_count.argtypes = [P]
    L.pamc_launch_count.restype = i64
    L.pamc_sweep_shape.argtypes = [P, P, P, P]
    L.pamc_weight_sum.argtypes = [P]
    L.pamc_weight_sum.restype = i64
    L.pamc_last_error.argtypes = [P, ctypes.c_char_p, ctypes.c_size_t]
    L.pamc_destroy.argtypes = [P]
    L.pamc_sweeps_noalloc.argtypes = [i32, i32, P, P, P, i32, i32, i32, i32, ctypes.c_double,
                                      ctypes.c_uint64, i32, P, P, P, P, ctypes.c_char_p,
                                      ctypes.c_size_t]
    L.pamc_dense_rows.argtypes = [P, P, P]
    L.pamc_control_history.argtypes = [P, P, P, P]
    L.pamc_sweep_mode.argtypes = [P, P]
    L.pamc_set_sweep_timing.argtypes = [P, ctypes.c_int]
    L.pamc_set_sweep_timing.restype = ctypes.c_int
    L.pamc_sweep_stats.argtypes = [P, P, P, P]
    L.pamc_sweep_stats.restype = ctypes.c_int
    L.pamc_sweep_mode.restype = ctypes.c_int
    L.pamc_control_history.restype = ctypes.c_int
    L.pamc_set_population.argtypes = [P, P]
    L.pamc_set_population.restype = ctypes.c_int
    L.pamc_fields.argtypes = [P, P]
    L.pamc_fields.restype = ctypes.c_int
    L.pamc_hamming.argtypes = [P, P, P]
    L.pamc_hamming.restype = ctypes.c_int
    L.pamc_lineage.argtypes = [P, P, P]
    L.pamc_lineage.restype = ctypes.c_int
    L.pamc_footprint.argtypes = [P, ctypes.POINTER(Params)]
    L.pamc_footprint.restype = ctypes.c_size_t
    L.pamc_batch_create.argtypes = [ctypes.c_int, P, ctypes.POINTER(P)]
    L.pamc_batch_add.argtypes = [P, P]
    L.pamc_batch_step.argtypes = [P, i32]
    L.pamc_batch_retire.argtypes = [P, P, i32]
    L.pamc_batch_retire.restype = i32
    for nm in ("pamc_batch_size", "pamc_batch_active"):
        getattr(L, nm).argtypes = [P]
        getattr(L, nm).restype = i32
    for nm in ("pamc_batch_launch_count", "pamc_batch_graph_builds"):
        getattr(L, nm).argtypes = [P]
        getattr(L, nm).restype = i64
    L.pamc_size_class.argtypes = [i32]
    L.pamc_size_class.restype = ctypes.c_int
    L.pamc_batch_set_shape.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.pamc_batch_set_shape.restype = ctypes.c_int
    L.pamc_batch_get_shape.argtypes = [P, ctypes.c_int, P, P]
    L.pamc_batch_get_shape.restype = ctypes.c_int
    L.pamc_batch_set_lanes.argtypes = [P, ctypes.c_int, ctypes.c_int]
    L.pamc_batch_set_lanes.restype = ctypes.c_int
    L.pamc_batch_get_lanes.argtypes = [P, ctypes.c_int, P]
    L.pamc_batch_get_lanes.restype = ctypes.c_int
    L.pamc_batch_set_placement.argtypes = [P, ctypes.c_int, ctypes.c_int]
    L.pamc_batch_set_placement.restype = ctypes.c_int
    L.pamc_batch_get_placement.argtypes = [P, ctypes.c_int, P]
    L.pamc_batch_get_placement.restype = ctypes.c_int
    L.pamc_batch_sync.argtypes = [P]
    L.pamc_batch_last_error.argtypes = [P, ctypes.c_char_p, ctypes.c_size_t]
    L.pamc_batch_destroy.argtypes = [P]
    L.pamc_batch_destroy.restype = None
    L.pamc_save.argtypes = [P, P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    L.pamc_load.argtypes = [P, P, ctypes.c_size_t]
    L.pamc_save.restype = ctypes.c_int
    L.pamc_load.restype = ctypes.c_int
    L.pamc_shard_range.argtypes = [i32, i32, i32, P, P]
    L.pamc_shard_init.argtypes = [P, ctypes.POINTER(Params), i32, i32]
    L.pamc_shard_energies.argtypes = [P, P]
    L.pamc_shard_resample.argtypes = [P, P, P]
    L.pamc_shard_plan.argtypes = [i32, i32, i32, P, P, P, P, P]
    L.pamc_shard_pack.argtypes = [P, P, i32, P]
    L.pamc_shard_sweep.argtypes = [P, P, P, P, i32, P]
    L.pamc_shard_control.argtypes = [P, P, P]
    L.pamc_shard_best.argtypes = [P, P, P, P]
    for nm in ("pamc_shard_range", "pamc_shard_init", "pamc_shard_energies", "pamc_shard_resample",
               "pamc_shard_plan", "pamc_shard_pack", "pamc_shard_sweep", "pamc_shard_control", "pamc_shard_best"):
        getattr(L, nm).restype = ctypes.c_int
    for nm in ("pamc_batch_create", "pamc_batch_add", "pamc_batch_step", "pamc_batch_sync",
               "pamc_batch_last_error"):
        getattr(L, nm).restype = ctypes.c_int
    for nm in ("pamc_sweeps_noalloc", "pamc_set_allocator", "pamc_create_csr", "pamc_create_dense", "pamc_init",
               "pamc_step", "pamc_sync", "pamc_run", "pamc_best", "pamc_state",
               "pamc_control_state", "pamc_last_error"):
        getattr(L, nm).restype = ctypes.c_int
    if torch_allocator:
        _register_torch_allocator(L)
    _lib = L
    return L


def _check(rc: int, h=None):
    if rc != 0:
        buf = ctypes.create_string_buffer(256)
        _lib.pamc_last_error(h, buf, 256)
        raise PamcError(rc, buf.value.decode(errors="replace"))


# handle address -> [n, R]: the sizes the library reads from or writes into
# caller buffers, so that a mismatched n or R is refused before a pointer is
# passed (handles made outside this module are not checked)
_dims = {}


def _dims_check(h, n=None, R=None):
    d = _dims.get(getattr(h, "value", None))
    if d is None:
        return
    if n is not None and int(n) != d[0]:
        raise ValueError(f"n = {int(n)} does not match the instance's n = {d[0]}")
    if R is not None and d[1] is not None and int(R) != d[1]:
        raise ValueError(f"R = {int(R)} does not match the population's R = {d[1]}")


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_ptr(device: int, stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    return ctypes.c_void_p(int(torch.cuda.current_stream(device).cuda_stream))


def make_params(**kw) -> Params:
    p = dict(DEFAULTS)
    p.update(kw)
    return Params(**p)


# ---------------------------------------------------------------- C-ABI mirror
def pamc_create_csr(n, row_ptr, col, w, device: int = 0, stream=None):
    L = load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32).reshape(-1)
    cl = np.ascontiguousarray(col, dtype=np.int32).reshape(-1)
    ww = np.ascontiguousarray(w, dtype=np.int32).reshape(-1)
    # the library reads n + 1 row pointers and row_ptr[n] entries of col and w
    if int(n) < 0 or rp.shape[0] != int(n) + 1:
        raise ValueError(f"row_ptr must hold n + 1 = {int(n) + 1} entries, got {rp.shape[0]}")
    nnz = int(rp[-1])
    if cl.shape[0] != nnz or ww.shape[0] != nnz:
        raise ValueError(f"col and w must hold row_ptr[n] = {nnz} entries, got {cl.shape[0]} and {ww.shape[0]}")
    h = ctypes.c_void_p()
    _check(L.pamc_create_csr(int(n), _ptr(rp), _ptr(cl), _ptr(ww), int(device),
                             _stream_ptr(device, stream), ctypes.byref(h)))
    _dims[h.value] = [int(n), None]
    return h


def pamc_create_dense(n, w, device: int = 0, stream=None):
    """w: host numpy int8 (n, n) or a CUDA tensor (pointer passed as device memory)."""
    L = load()
    h = ctypes.c_void_p()
    if tuple(w.shape) != (int(n), int(n)):
        raise ValueError(f"w must be n x n = ({int(n)}, {int(n)}), got {tuple(w.shape)}")
    if isinstance(w, np.ndarray):
        arr = np.ascontiguousarray(w, dtype=np.int8)
        _check(L.pamc_create_dense(int(n), _ptr(arr), 0, int(device), _stream_ptr(device, stream),
                                   ctypes.byref(h)))
    else:
        import torch
        if w.dtype != torch.int8 or not w.is_cuda or not w.is_contiguous():
            raise ValueError("a device w must be a contiguous CUDA int8 tensor")
        _check(L.pamc_create_dense(int(n), ctypes.c_void_p(int(w.data_ptr())), 1, int(device),
                                   _stream_ptr(device, stream), ctypes.byref(h)))
    _dims[h.value] = [int(n), None]
    return h


def _set_R(h, R):
    d = _dims.get(getattr(h, "value", None))
    if d is not None:
        _dims[h.value] = [d[0], int(R)]


def pamc_init(h, **params):
    p = make_params(**params)
    _check(_lib.pamc_init(h, ctypes.byref(p)), h)
    _set_R(h, p.R)
    return p


def pamc_step(h, nsteps: int = 1):
    _check(_lib.pamc_step(h, int(nsteps)), h)


def pamc_sync(h):
    _check(_lib.pamc_sync(h), h)


def pamc_run(h, **params):
    p = make_params(**params)
    _check(_lib.pamc_run(h, ctypes.byref(p)), h)
    _set_R(h, p.R)
    return p


def pamc_best(h, n: int):
    _dims_check(h, n=n)
    cut = np.zeros(1, dtype=np.int64)
    spins = np.zeros(n, dtype=np.int8)
    _check(_lib.pamc_best(h, _ptr(cut), _ptr(spins)), h)
    return int(cut[0]), spins


def pamc_state(h, R: int, n: int):
    _dims_check(h, n=n, R=R)
    spins = np.zeros((R, n), dtype=np.int8)
    E = np.zeros(R, dtype=np.int64)
    par = np.zeros(R, dtype=np.int32)
    cnt = np.zeros(R, dtype=np.int32)
    _check(_lib.pamc_state(h, _ptr(spins), _ptr(E), _ptr(par), _ptr(cnt)), h)
    return spins, E, par, cnt


CTL_KEYS = ("t", "z", "cycle", "cooldown", "enable_cm", "done", "ncm_last", "hist_len",
            "ncm_flipped", "ncm_dE_max")


def pamc_control_state(h) -> dict:
    iv = np.zeros(10, dtype=np.int64)
    dv = np.zeros(2, dtype=np.float64)
    _check(_lib.pamc_control_state(h, _ptr(iv), _ptr(dv)), h)
    d = {k: int(v) for k, v in zip(CTL_KEYS, iv)}
    d["beta"], d["delta"] = float(dv[0]), float(dv[1])
    return d


def pamc_control_history(h):
    """(history of M*, oldest first, as an int64 array; M* so far)."""
    hist = np.zeros(64, dtype=np.int64)
    ln = np.zeros(1, dtype=np.int32)
    m = np.zeros(1, dtype=np.int64)
    _check(_lib.pamc_control_history(h, _ptr(hist), _ptr(ln), _ptr(m)), h)
    return hist[:int(ln[0])].copy(), int(m[0])


def pamc_launch_count(h) -> int:
    return int(_lib.pamc_launch_count(h))


def pamc_dense_rows(h) -> tuple:
    """(coupling rows gathered by the dense field updates, positions visited) since pamc_init."""
    v = np.zeros(2, dtype=np.int64)
    _check(_lib.pamc_dense_rows(h, _ptr(v[0:1]), _ptr(v[1:2])), h)
    return int(v[0]), int(v[1])


def pamc_sweep_shape(h) -> tuple:
    """(groups per CTA, warps per group, lanes per vertex) of the sparse sweep."""
    v = np.zeros(3, dtype=np.int32)
    _check(_lib.pamc_sweep_shape(h, _ptr(v[0:1]), _ptr(v[1:2]), _ptr(v[2:3])), h)
    return int(v[0]), int(v[1]), int(v[2])


def pamc_sweep_mode(h) -> int:
    """0 pull over CSR rows, 1 pull over ELL rows, 2 push (fields kept and updated on flips)."""
    v = ctypes.c_int(0)
    _check(_lib.pamc_sweep_mode(h, ctypes.byref(v)), h)
    return v.value


def pamc_set_sweep_timing(h, on: bool = True):
    _check(_lib.pamc_set_sweep_timing(h, 1 if on else 0), h)


def pamc_sweep_stats(h) -> dict:
    """flips since init; launches and ms of the sweep launches timed since the last call."""
    f = np.zeros(2, dtype=np.int64)
    ms = np.zeros(1, dtype=np.float64)
    _check(_lib.pamc_sweep_stats(h, _ptr(f[0:1]), _ptr(f[1:2]), _ptr(ms)), h)
    return {"flips": int(f[0]), "launches": int(f[1]), "ms": float(ms[0])}


def pamc_weight_sum(h) -> int:
    return int(_lib.pamc_weight_sum(h))


def pamc_last_error(h=None) -> str:
    buf = ctypes.create_string_buffer(256)
    load().pamc_last_error(h, buf, 256)
    return buf.value.decode(errors="replace")


def pamc_destroy(h):
    if h is not None and h.value:
        _dims.pop(h.value, None)
        _lib.pamc_destroy(h)


def pamc_sweeps_noalloc(n, nnz, row_ptr, col, w, H, rule, R, sweeps, beta, seed, t, spins_in,
                        spins_out, E_out, stream=None):
    """S sweeps at a fixed beta on a caller-owned device population without any
    allocation by the library.  Every array argument is a CUDA tensor or a raw
    device address (int); see include/pamc.h for the contract.  Tensors are
    checked before any pointer is passed: one CUDA device for all of them,
    contiguous, int32 CSR arrays of n + 1 and nnz entries, int8 spins of at
    least R * n and int64 energies of at least R; the call runs with that
    device current."""
    L = load()
    # sizes beyond the library's limits are refused by the library itself,
    # before it reads any pointer; tensor sizes are checked only within them
    in_limits = (1 <= int(n) <= NOALLOC_MAX_N and 0 <= int(nnz) <= NOALLOC_MAX_NNZ
                 and 1 <= int(R) <= NOALLOC_MAX_R and 0 <= int(sweeps) <= NOALLOC_MAX_SWEEPS)
    want = {"row_ptr": (row_ptr, "int32", int(n) + 1), "col": (col, "int32", int(nnz)),
            "w": (w, "int32", int(nnz)), "spins_in": (spins_in, "int8", int(R) * int(n)),
            "spins_out": (spins_out, "int8", int(R) * int(n)), "E_out": (E_out, "int64", int(R))}
    dev = None
    for name, (x, dt, count) in want.items():
        if x is None or isinstance(x, int):
            continue
        if not getattr(x, "is_cuda", False):
            raise ValueError(f"{name} must be a CUDA tensor or a device address")
        if str(x.dtype) != "torch." + dt:
            raise ValueError(f"{name} must be {dt}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if in_limits and x.numel() < count:
            raise ValueError(f"{name} holds {x.numel()} elements, the call reads or writes {count}")
        d = x.device.index or 0
        if dev is not None and d != dev:
            raise ValueError(f"{name} is on cuda:{d}, other arguments on cuda:{dev}")
        dev = d

    def addr(x):
        if x is None:
            return None
        return ctypes.c_void_p(int(x) if isinstance(x, int) else int(x.data_ptr()))

    def call():
        d = dev if dev is not None else 0
        buf = ctypes.create_string_buffer(256)
        rc = L.pamc_sweeps_noalloc(int(n), int(nnz), addr(row_ptr), addr(col), addr(w), int(H),
                                   int(rule), int(R), int(sweeps), float(beta), int(seed), int(t),
                                   addr(spins_in), addr(spins_out), addr(E_out),
                                   _stream_ptr(d, stream), buf, 256)
        if rc != 0:
            raise PamcError(rc, buf.value.decode(errors="replace"))

    if dev is None:
        call()
        return
    import torch
    with torch.cuda.device(dev):
        call()


# ---------------------------------------------------------------- checkpoints
def pamc_save(h) -> bytes:
    """The run's whole state at the start of its next iteration (see
    include/pamc.h)."""
    size = ctypes.c_size_t(0)
    _check(_lib.pamc_save(h, None, 0, ctypes.byref(size)), h)
    buf = ctypes.create_string_buffer(size.value)
    _check(_lib.pamc_save(h, buf, size.value, ctypes.byref(size)), h)
    return buf.raw[:size.value]


def pamc_load(h, data: bytes):
    """Continue a run from pamc_save's bytes on a handle of the same instance."""
    raw = bytes(data)
    buf = ctypes.create_string_buffer(raw, len(raw))
    _check(_lib.pamc_load(h, buf, len(raw)), h)
    d = _dims.get(getattr(h, "value", None))
    if d is not None:
        _dims[h.value] = [d[0], None]   # R comes from the checkpoint


# ---------------------------------------------------------------- split population
def _dev_arg(x, name, dtype, count, allow_none=False):
    """A contiguous CUDA tensor of dtype holding at least count elements ->
    its device address."""
    if x is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not getattr(x, "is_cuda", False):
        raise ValueError(f"{name} must be a CUDA tensor")
    if str(x.dtype) != "torch." + dtype:
        raise ValueError(f"{name} must be {dtype}, got {x.dtype}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if x.numel() < count:
        raise ValueError(f"{name} holds {x.numel()} elements, the call uses {count}")
    return ctypes.c_void_p(int(x.data_ptr()))


def _shard_dims(h):
    d = _dims.get(getattr(h, "value", None))
    if d is None or len(d) < 4:
        raise ValueError("not a split-population handle made by pamc_shard_init")
    return d   # [n, own count, R, nranks]


def pamc_shard_range(R: int, nranks: int, rank: int):
    """(base, count): the own slots of process rank (host only)."""
    L = load(torch_allocator=False)
    b = np.zeros(1, dtype=np.int32)
    c = np.zeros(1, dtype=np.int32)
    rc = L.pamc_shard_range(int(R), int(nranks), int(rank), _ptr(b), _ptr(c))
    if rc != 0:
        raise PamcError(rc, "R must be a multiple of 4 nranks and 0 <= rank < nranks")
    return int(b[0]), int(c[0])


def pamc_shard_init(h, rank: int, nranks: int, **params):
    p = make_params(**params)
    _check(_lib.pamc_shard_init(h, ctypes.byref(p), int(rank), int(nranks)), h)
    d = _dims.get(getattr(h, "value", None))
    if d is not None:
        _, count = pamc_shard_range(p.R, nranks, rank)
        _dims[h.value] = [d[0], count, int(p.R), int(nranks)]
    return p


def pamc_shard_energies(h, E_own):
    _, c, _, _ = _shard_dims(h)
    _check(_lib.pamc_shard_energies(h, _dev_arg(E_own, "E_own", "int64", c)), h)


def pamc_shard_resample(h, E_all) -> np.ndarray:
    _, _, R, _ = _shard_dims(h)
    parent = np.zeros(R, dtype=np.int32)
    _check(_lib.pamc_shard_resample(h, _dev_arg(E_all, "E_all", "int64", R), _ptr(parent)), h)
    return parent


def pamc_shard_plan(R: int, nranks: int, rank: int, parent):
    """(send_counts, send_rows, recv_counts, local_parent) for process rank
    (host only; see include/pamc.h)."""
    L = load(torch_allocator=False)
    par = np.ascontiguousarray(parent, dtype=np.int32).reshape(-1)
    if par.shape[0] != int(R):
        raise ValueError(f"parent must hold R = {int(R)} entries, got {par.shape[0]}")
    _, c = pamc_shard_range(R, nranks, rank)
    sc = np.zeros(int(nranks), dtype=np.int32)
    rc_ = np.zeros(int(nranks), dtype=np.int32)
    rows = np.zeros(max(int(R) - c, 1), dtype=np.int32)
    lp = np.zeros(c, dtype=np.int32)
    rc = L.pamc_shard_plan(int(R), int(nranks), int(rank), _ptr(par), _ptr(sc), _ptr(rows), _ptr(rc_), _ptr(lp))
    if rc != 0:
        raise PamcError(rc, "pamc_shard_plan: parent entries must lie in [0, R)")
    return sc, rows[:int(sc.sum())].copy(), rc_, lp


def pamc_shard_pack(h, rows, sendbuf):
    n, c, R, _ = _shard_dims(h)
    r = np.ascontiguousarray(rows, dtype=np.int32).reshape(-1)
    k = int(r.shape[0])
    buf = _dev_arg(sendbuf, "sendbuf", "int8", k * n) if k > 0 else None
    _check(_lib.pamc_shard_pack(h, _ptr(r) if k > 0 else None, k, buf), h)


def pamc_shard_sweep(h, E_all, local_parent, imports, nimports: int, E_own=None):
    n, c, R, _ = _shard_dims(h)
    lp = np.ascontiguousarray(local_parent, dtype=np.int32).reshape(-1)
    if lp.shape[0] != c:
        raise ValueError(f"local_parent must hold the {c} own slots, got {lp.shape[0]}")
    k = int(nimports)
    imp = _dev_arg(imports, "imports", "int8", k * n) if k > 0 else None
    _check(_lib.pamc_shard_sweep(h, _dev_arg(E_all, "E_all", "int64", R), _ptr(lp), imp, k,
                                 _dev_arg(E_own, "E_own", "int64", c, allow_none=True)), h)


def pamc_shard_control(h, E_all, E_own=None):
    _, c, R, _ = _shard_dims(h)
    _check(_lib.pamc_shard_control(h, _dev_arg(E_all, "E_all", "int64", R),
                                   _dev_arg(E_own, "E_own", "int64", c, allow_none=True)), h)


def pamc_shard_best(h):
    """(cut, spins or None, owned): M* and, on the process holding it, its
    configuration."""
    n = _shard_dims(h)[0]
    cut = np.zeros(1, dtype=np.int64)
    owned = np.zeros(1, dtype=np.int32)
    spins = np.zeros(n, dtype=np.int8)
    _check(_lib.pamc_shard_best(h, _ptr(cut), _ptr(spins), _ptr(owned)), h)
    return int(cut[0]), (spins if owned[0] else None), bool(owned[0])


def pamc_set_population(h, spins):
    arr = np.ascontiguousarray(spins, dtype=np.int8)
    d = _dims.get(getattr(h, "value", None))
    if d is not None and d[1] is not None and arr.size != d[0] * d[1]:
        raise ValueError(f"spins must hold R x n = {d[1]} x {d[0]} values, got {arr.size}")
    _check(_lib.pamc_set_population(h, _ptr(arr)), h)


def pamc_fields(h, R: int, n: int):
    _dims_check(h, n=n, R=R)
    H = np.zeros((R, n), dtype=np.int32)
    _check(_lib.pamc_fields(h, _ptr(H)), h)
    return H


def pamc_hamming(h, n: int):
    """(hist, sum): hist[k] = pairs of replicas at corrected distance k = min(d, n - d)."""
    _dims_check(h, n=n)
    hist = np.zeros(n // 2 + 1, dtype=np.int64)
    total = np.zeros(1, dtype=np.int64)
    _check(_lib.pamc_hamming(h, _ptr(hist), _ptr(total)), h)
    return hist, int(total[0])


def pamc_lineage(h, R: int):
    """(family, n_families): family[r] = the initial slot that slot r descends from."""
    _dims_check(h, R=R)
    fam = np.zeros(R, dtype=np.int32)
    k = np.zeros(1, dtype=np.int32)
    _check(_lib.pamc_lineage(h, _ptr(fam), _ptr(k)), h)
    return fam, int(k[0])


def pamc_footprint(h, **params) -> int:
    return int(_lib.pamc_footprint(h, ctypes.byref(make_params(**params))))


def _bcheck(rc: int, b=None):
    if rc != 0:
        buf = ctypes.create_string_buffer(256)
        _lib.pamc_batch_last_error(b, buf, 256)
        raise PamcError(rc, buf.value.decode(errors="replace"))


def pamc_batch_create(device: int = 0, stream=None):
    """stream None: the batch creates its own non-blocking stream."""
    L = load()
    b = ctypes.c_void_p()
    st = ctypes.c_void_p(int(stream)) if stream is not None else None
    _bcheck(L.pamc_batch_create(int(device), st, ctypes.byref(b)))
    return b


def pamc_batch_add(b, h):
    _bcheck(_lib.pamc_batch_add(b, h), b)


def pamc_batch_step(b, nsteps: int = 1):
    _bcheck(_lib.pamc_batch_step(b, int(nsteps)), b)


def pamc_batch_retire(b, max_out: int = 4096) -> list:
    out = (ctypes.c_void_p * max(int(max_out), 1))()
    k = _lib.pamc_batch_retire(b, out, int(max_out))
    if k < 0:
        _bcheck(int(STATUS_CODES["PAMC_ERR_CUDA"]), b)
    return [ctypes.c_void_p(out[i]) for i in range(k)]


def pamc_size_class(n: int) -> int:
    return int(load().pamc_size_class(int(n)))


def pamc_batch_set_shape(b, size_class: int, groups_per_cta: int, warps_per_group: int):
    _bcheck(_lib.pamc_batch_set_shape(b, int(size_class), int(groups_per_cta), int(warps_per_group)), b)


def pamc_batch_get_shape(b, size_class: int):
    g, w = ctypes.c_int(0), ctypes.c_int(0)
    _bcheck(_lib.pamc_batch_get_shape(b, int(size_class), ctypes.byref(g), ctypes.byref(w)), b)
    return g.value, w.value


def pamc_batch_set_lanes(b, size_class: int, lanes_per_vertex: int):
    _bcheck(_lib.pamc_batch_set_lanes(b, int(size_class), int(lanes_per_vertex)), b)


def pamc_batch_get_lanes(b, size_class: int) -> int:
    v = ctypes.c_int(0)
    _bcheck(_lib.pamc_batch_get_lanes(b, int(size_class), ctypes.byref(v)), b)
    return v.value


def pamc_batch_set_placement(b, size_class: int, global_spins: bool):
    """Spin words of the class's Ising groups in device memory (True) or shared memory (False)."""
    _bcheck(_lib.pamc_batch_set_placement(b, int(size_class), 1 if global_spins else 0), b)


def pamc_batch_get_placement(b, size_class: int) -> bool:
    v = ctypes.c_int(0)
    _bcheck(_lib.pamc_batch_get_placement(b, int(size_class), ctypes.byref(v)), b)
    return bool(v.value)


def pamc_batch_size(b) -> int:
    return int(_lib.pamc_batch_size(b))


def pamc_batch_active(b) -> int:
    return int(_lib.pamc_batch_active(b))


def pamc_batch_launch_count(b) -> int:
    return int(_lib.pamc_batch_launch_count(b))


def pamc_batch_graph_builds(b) -> int:
    return int(_lib.pamc_batch_graph_builds(b))


def pamc_batch_sync(b):
    _bcheck(_lib.pamc_batch_sync(b), b)


def pamc_batch_destroy(b):
    if b is not None and b.value:
        _lib.pamc_batch_destroy(b)


class Solver:
    """Convenience owner of one handle on a CSR Max-Cut instance."""

    def __init__(self, row_ptr, col, w, device: int = 0, stream=None):
        self.n = len(row_ptr) - 1
        self.h = pamc_create_csr(self.n, row_ptr, col, w, device, stream)
        self.R = 0

    def init(self, **params):
        p = pamc_init(self.h, **params)
        self.R = p.R
        return p

    def step(self, k: int = 1):
        pamc_step(self.h, k)

    def sync(self):
        pamc_sync(self.h)

    def run(self, **params):
        p = pamc_run(self.h, **params)
        self.R = p.R
        return p

    def best(self):
        return pamc_best(self.h, self.n)

    def state(self):
        return pamc_state(self.h, self.R, self.n)

    def control(self):
        return pamc_control_state(self.h)

    def launches(self) -> int:
        return pamc_launch_count(self.h)

    def save(self) -> bytes:
        """Checkpoint of the run (pamc_save)."""
        return pamc_save(self.h)

    def load(self, data: bytes, R: int):
        """Continue from a checkpoint of this instance (pamc_load); R is the
        checkpointed run's population size."""
        pamc_load(self.h, data)
        self.R = int(R)
        _set_R(self.h, R)

    def close(self):
        pamc_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            if self.h is not None:
                self.close()
        except Exception:
            pass
