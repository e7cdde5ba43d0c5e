"""CPU oracle for augmented Population Annealing Monte Carlo.

TEST INFRASTRUCTURE ONLY.  This package is the independent checker of the CUDA
path: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (``--impl reference`` and the ``cpu_baseline`` object) may import it.  The
product package never imports it, and it imports nothing from the product.

The arithmetic lives in ``pamc_oracle.c`` (plain single-threaded C, binary64,
built with ``-ffp-contract=off``); this module only compiles it and marshals
numpy arrays through ctypes.  See ``pamc_oracle.h`` for the paper passage each
function follows.

Every function is pinned (``tests/test_oracle_pins*.py``); the NCM defaults,
the reading that a restart re-draws the population and the Potts beta factor
of Eq. 8 are readings of the paper, stated beside the functions that take them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pamc_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liborc.so")
_lock = threading.Lock()
_lib = None

TAG_INIT, TAG_PERM, TAG_FLIP, TAG_RESAMPLE, TAG_NCM = 1, 2, 3, 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (no GPU, no CUDA)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    hdr = os.path.join(_HERE, "pamc_oracle.h")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("rule", ctypes.c_int32),
        ("R", ctypes.c_int32), ("sweeps", ctypes.c_int32), ("steps", ctypes.c_int32),
        ("beta0", ctypes.c_double), ("beta1", ctypes.c_double),
        ("stagnation", ctypes.c_int32), ("z_rst", ctypes.c_int32),
        ("cooldown_tau", ctypes.c_int32), ("n_top", ctypes.c_int32), ("mis_trials", ctypes.c_int32),
        ("win_short", ctypes.c_int32), ("win_long", ctypes.c_int32),
        ("max_distinct_short", ctypes.c_int32), ("max_distinct_long", ctypes.c_int32),
        ("reheat_factor", ctypes.c_double), ("target_cut", ctypes.c_int64),
        ("seed", ctypes.c_uint64), ("restart_reinit", ctypes.c_int32), ("resample", ctypes.c_int32),
        ("K", ctypes.c_int32), ("gamma", ctypes.c_double),
    ]


class _Ctl(ctypes.Structure):
    _fields_ = [("z", ctypes.c_int32), ("cycle", ctypes.c_int32), ("cooldown", ctypes.c_int32),
                ("enable_cm", ctypes.c_int32), ("hist_len", ctypes.c_int32),
                ("beta", ctypes.c_double), ("delta", ctypes.c_double),
                ("hist", ctypes.c_int64 * 64)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # PAMC_ORACLE_LIB: a test-built variant of this library (the
            # mutation tests build copies of the oracle with a planted mistake
            # and check that the pins reject them)
            path = os.environ.get("PAMC_ORACLE_LIB") or build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            L.orc_philox4x32_10.argtypes = [P, P, P]
            L.orc_det_exp.argtypes = [dbl]; L.orc_det_exp.restype = dbl
            L.orc_round_nonneg.argtypes = [dbl]; L.orc_round_nonneg.restype = u64
            L.orc_thr_heatbath.argtypes = [dbl, i64]; L.orc_thr_heatbath.restype = u64
            L.orc_thr_metropolis.argtypes = [dbl, i64]; L.orc_thr_metropolis.restype = u64
            L.orc_thr_potts_b1.argtypes = [dbl, i64, i64]; L.orc_thr_potts_b1.restype = u64
            L.orc_thr_potts_b2.argtypes = [dbl, i64]; L.orc_thr_potts_b2.restype = u64
            L.orc_permutation.argtypes = [i32, u64, i32, i32, P]
            L.orc_resample.argtypes = [i32, P, dbl, dbl, u64, i32, P, P]; L.orc_resample.restype = ctypes.c_int
            L.orc_create.argtypes = [i32, P, P, P, ctypes.POINTER(_Params)]; L.orc_create.restype = P
            L.orc_destroy.argtypes = [P]
            L.orc_step.argtypes = [P, i32]; L.orc_step.restype = i32
            for nm in ("orc_get_spins", "orc_get_fields", "orc_get_energy"):
                getattr(L, nm).argtypes = [P, P]
            L.orc_get_parents.argtypes = [P, P, P]
            L.orc_get_best.argtypes = [P, P, P]
            L.orc_get_ctl.argtypes = [P, P, P]
            L.orc_weight_sum.argtypes = [P]; L.orc_weight_sum.restype = i64
            L.orc_set_spins.argtypes = [P, P]
            L.orc_energy_ising.argtypes = [i32, P, P, P, P]; L.orc_energy_ising.restype = i64
            L.orc_energy_potts.argtypes = [i32, P, P, P, P]; L.orc_energy_potts.restype = i64
            L.orc_ncm_replica.argtypes = [i32, P, P, P, P, P, i32, u64, i32, i32]
            L.orc_ncm_replica.restype = i32
            L.orc_control.argtypes = [ctypes.POINTER(_Ctl), ctypes.POINTER(_Params), dbl, i64]
            L.orc_control.restype = ctypes.c_int
            L.orc_softmax_pick.argtypes = [i32, P, dbl, dbl, P]
            L.orc_softmax_pick.restype = i32
            L.orc_set_state.argtypes = [P, i32, ctypes.POINTER(_Ctl), i64, P, P]
            L.orc_set_sweep_replay.argtypes = [P, P, P]
            L.orc_get_ncm_targets.argtypes = [P, P, P]
            L.orc_get_history.argtypes = [P, P]
            L.orc_sweep_flips.argtypes = [P]
            L.orc_sweep_flips.restype = i64
            for nm in ("orc_iter_population", "orc_iter_sweeps", "orc_iter_control"):
                getattr(L, nm).argtypes = [P]
                getattr(L, nm).restype = None
            L.orc_set_own.argtypes = [P, i32, i32]
            L.orc_set_energies.argtypes = [P, P]
            L.orc_set_rows.argtypes = [P, i32, i32, P]
            L.orc_best_owned.argtypes = [P]
            L.orc_best_owned.restype = i32
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- primitives
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def det_exp(x: float) -> float:
    return lib().orc_det_exp(float(x))


def round_nonneg(x: float) -> int:
    return int(lib().orc_round_nonneg(float(x)))


def thr_heatbath(beta: float, h: int) -> int:
    return int(lib().orc_thr_heatbath(float(beta), int(h)))


def thr_metropolis(beta: float, dE: int) -> int:
    return int(lib().orc_thr_metropolis(float(beta), int(dE)))


def thr_potts_b1(beta: float, a: int, b: int) -> int:
    return int(lib().orc_thr_potts_b1(float(beta), int(a), int(b)))


def thr_potts_b2(beta: float, c: int) -> int:
    return int(lib().orc_thr_potts_b2(float(beta), int(c)))


def permutation(n: int, seed: int, t: int, sweep: int) -> np.ndarray:
    out = np.zeros(max(n, 1), dtype=np.int32)
    lib().orc_permutation(int(n), int(seed), int(t), int(sweep), _ptr(out))
    return out[:n]


def resample(E, delta: float, escale: float, seed: int, t: int):
    E = np.ascontiguousarray(np.asarray(E, dtype=np.int64))
    R = E.shape[0]
    parent = np.zeros(R, dtype=np.int32)
    count = np.zeros(R, dtype=np.int32)
    rc = lib().orc_resample(R, _ptr(E), float(delta), float(escale), int(seed), int(t),
                            _ptr(parent), _ptr(count))
    if rc != 0:
        raise ValueError("resample failed")
    return parent, count


def energy_ising(rp, col, J, s) -> int:
    rp, col, J = (np.ascontiguousarray(x, dtype=np.int32) for x in (rp, col, J))
    s = np.ascontiguousarray(s, dtype=np.int8)
    return int(lib().orc_energy_ising(len(rp) - 1, _ptr(rp), _ptr(col), _ptr(J), _ptr(s)))


def energy_potts(rp, col, J, s) -> int:
    rp, col, J = (np.ascontiguousarray(x, dtype=np.int32) for x in (rp, col, J))
    s = np.ascontiguousarray(s, dtype=np.int8)
    return int(lib().orc_energy_potts(len(rp) - 1, _ptr(rp), _ptr(col), _ptr(J), _ptr(s)))


def ncm_replica(rp, col, J, s, h, mis_trials, seed, t, r):
    """Non-local cluster move on one replica (in place); returns #flipped."""
    rp, col, J = (np.ascontiguousarray(x, dtype=np.int32) for x in (rp, col, J))
    assert s.dtype == np.int8 and h.dtype == np.int32
    return int(lib().orc_ncm_replica(len(rp) - 1, _ptr(rp), _ptr(col), _ptr(J), _ptr(s), _ptr(h),
                                     int(mis_trials), int(seed), int(t), int(r)))


def softmax_pick(syn, beta: float, gamma: float, u) -> int:
    """One softmax noisy-argmax label choice (see pamc_oracle.h)."""
    syn = np.ascontiguousarray(syn, dtype=np.int32)
    u = np.ascontiguousarray(u, dtype=np.uint32)
    return int(lib().orc_softmax_pick(int(syn.shape[0]), _ptr(syn), float(beta), float(gamma), _ptr(u)))


def hamming_counts(spins):
    """Replica diversity (Suppl., Hamming distance of replicas), written out
    from its definition: for every pair r < r' of the R x n +-1 population,
    d = the number of spins in which the two replicas differ, corrected for the
    global flip symmetry as dc = min(d, n - d).  Returns (hist, total) with
    hist[k] = the number of pairs with dc = k (k = 0 .. n // 2) and total = the
    sum of dc over all pairs."""
    spins = np.asarray(spins)
    R, n = spins.shape
    hist = np.zeros(n // 2 + 1, dtype=np.int64)
    total = 0
    for r in range(R):
        for q in range(r + 1, R):
            d = int(np.count_nonzero(spins[r] != spins[q]))
            dc = min(d, n - d)
            hist[dc] += 1
            total += dc
    return hist, total


def lineage_step(family, parent, reinitialised: bool = False):
    """Genealogy through one population step: slot m inherits its resampling
    parent's family; a re-initialised population starts new families."""
    family = np.asarray(family)
    if reinitialised:
        return np.arange(family.shape[0], dtype=family.dtype)
    return family[np.asarray(parent)]


class Controller:
    """Algorithm 1's post-sweep control block on its own (for hand-built M*
    sequences): ``update(mstar)`` returns True when the schedule restarts."""

    def __init__(self, **params):
        self.p = make_params(**params)
        self._p = _Params(**self.p)
        self.dbeta = ((self.p["beta1"] - self.p["beta0"]) / (self.p["steps"] - 1)
                      if self.p["steps"] > 1 else 0.0)
        self.c = _Ctl(z=1, cycle=0, cooldown=0, enable_cm=0, hist_len=0,
                      beta=self.p["beta0"], delta=self.dbeta)

    def update(self, mstar: int) -> bool:
        return bool(lib().orc_control(ctypes.byref(self.c), ctypes.byref(self._p),
                                      float(self.dbeta), int(mstar)))

    def state(self) -> dict:
        c = self.c
        return dict(z=c.z, cycle=c.cycle, cooldown=c.cooldown, enable_cm=c.enable_cm,
                    hist_len=c.hist_len, beta=c.beta, delta=c.delta)


# ---------------------------------------------------------------- full runs
DEFAULTS = dict(kind=0, rule=0, R=16, sweeps=1, steps=10, beta0=0.1, beta1=3.0, stagnation=0,
                z_rst=0, cooldown_tau=10, n_top=0, mis_trials=4, win_short=25, win_long=40,
                max_distinct_short=3, max_distinct_long=5, reheat_factor=0.8, target_cut=-1,
                seed=0, restart_reinit=1, resample=1, K=3, gamma=1.0)


def make_params(**kw) -> dict:
    p = dict(DEFAULTS)
    p.update(kw)
    if p["n_top"] <= 0:
        p["n_top"] = max(1, p["R"] // 16)
    return p


class OracleRun:
    """One Algorithm 1 run on a CSR Max-Cut instance (weights w)."""

    def __init__(self, row_ptr, col, w, **params):
        self.p = make_params(**params)
        self.rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.w = np.ascontiguousarray(w, dtype=np.int32)
        self.n = len(self.rp) - 1
        cp = _Params(**self.p)
        self._h = lib().orc_create(self.n, _ptr(self.rp), _ptr(self.col), _ptr(self.w), ctypes.byref(cp))
        if not self._h:
            raise ValueError("oracle rejected the instance or parameters")

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def step(self, k: int = 1) -> int:
        return int(lib().orc_step(self._h, int(k)))

    @property
    def R(self):
        return self.p["R"]

    def spins(self) -> np.ndarray:
        out = np.zeros((self.R, self.n), dtype=np.int8)
        lib().orc_get_spins(self._h, _ptr(out))
        return out

    def fields(self) -> np.ndarray:
        f = self.p["K"] if self.p["kind"] == 1 else 1
        out = np.zeros((self.R, self.n * f), dtype=np.int32)
        lib().orc_get_fields(self._h, _ptr(out))
        return out.reshape(self.R, self.n, f) if self.p["kind"] == 1 else out

    def energy(self) -> np.ndarray:
        out = np.zeros(self.R, dtype=np.int64)
        lib().orc_get_energy(self._h, _ptr(out))
        return out

    def parents(self):
        par = np.zeros(self.R, dtype=np.int32)
        cnt = np.zeros(self.R, dtype=np.int32)
        lib().orc_get_parents(self._h, _ptr(par), _ptr(cnt))
        return par, cnt

    def best(self):
        m = np.zeros(1, dtype=np.int64)
        s = np.zeros(self.n, dtype=np.int8)
        lib().orc_get_best(self._h, _ptr(m), _ptr(s))
        return int(m[0]), s

    def ctl(self) -> dict:
        iv = np.zeros(10, dtype=np.int64)
        dv = np.zeros(2, dtype=np.float64)
        lib().orc_get_ctl(self._h, _ptr(iv), _ptr(dv))
        keys = ("t", "z", "cycle", "cooldown", "enable_cm", "done", "ncm_last", "hist_len",
                "ncm_flipped", "ncm_dE_max")
        d = {k: int(v) for k, v in zip(keys, iv)}
        d["beta"], d["delta"] = float(dv[0]), float(dv[1])
        return d

    def weight_sum(self) -> int:
        return int(lib().orc_weight_sum(self._h))

    def set_spins(self, s: np.ndarray):
        s = np.ascontiguousarray(s, dtype=np.int8).reshape(self.R, self.n)
        lib().orc_set_spins(self._h, _ptr(s))

    def set_state(self, t: int, ctl: dict, hist, mstar: int, best, spins):
        """Load a state of Algorithm 1 reached elsewhere (see orc_set_state):
        ctl holds z, cycle, cooldown, enable_cm, beta and delta; hist the M*
        history, oldest first."""
        hist = np.asarray(hist, dtype=np.int64).reshape(-1)
        c = _Ctl(z=int(ctl["z"]), cycle=int(ctl["cycle"]), cooldown=int(ctl["cooldown"]),
                 enable_cm=int(ctl["enable_cm"]), hist_len=int(hist.shape[0]), beta=float(ctl["beta"]),
                 delta=float(ctl["delta"]))
        for i, v in enumerate(hist.tolist()):
            c.hist[i] = int(v)
        sp = np.ascontiguousarray(spins, dtype=np.int8).reshape(self.R, self.n)
        b = None if best is None else _ptr(np.ascontiguousarray(best, dtype=np.int8).reshape(self.n))
        lib().orc_set_state(self._h, int(t), ctypes.byref(c), int(mstar), b, _ptr(sp))

    def set_sweep_replay(self, mask=None, spins_after=None):
        """Sweep only the replicas in mask; the others take spins_after (see
        orc_set_sweep_replay).  No arguments: every replica is swept again."""
        if mask is None:
            lib().orc_set_sweep_replay(self._h, None, None)
            return
        m = np.ascontiguousarray(np.asarray(mask, dtype=bool).astype(np.uint8).reshape(self.R))
        sa = np.ascontiguousarray(spins_after, dtype=np.int8).reshape(self.R, self.n)
        lib().orc_set_sweep_replay(self._h, _ptr(m), _ptr(sa))

    def sweep_flips(self) -> int:
        return int(lib().orc_sweep_flips(self._h))

    def history(self) -> np.ndarray:
        out = np.zeros(64, dtype=np.int64)
        lib().orc_get_history(self._h, _ptr(out))
        return out[:self.ctl()["hist_len"]]

    # one population split over several processes (orc_set_own and the
    # three parts of an iteration; see pamc_oracle.h)
    def iter_population(self):
        lib().orc_iter_population(self._h)

    def iter_sweeps(self):
        lib().orc_iter_sweeps(self._h)

    def iter_control(self):
        lib().orc_iter_control(self._h)

    def set_own(self, lo: int, hi: int):
        lib().orc_set_own(self._h, int(lo), int(hi))

    def set_energies(self, E):
        e = np.ascontiguousarray(E, dtype=np.int64).reshape(self.R)
        lib().orc_set_energies(self._h, _ptr(e))

    def set_rows(self, r0: int, rows):
        rw = np.ascontiguousarray(rows, dtype=np.int8).reshape(-1, self.n)
        lib().orc_set_rows(self._h, int(r0), int(rw.shape[0]), _ptr(rw))

    def best_owned(self) -> bool:
        return bool(lib().orc_best_owned(self._h))

    def ncm_targets(self) -> np.ndarray:
        out = np.zeros(self.R, dtype=np.int32)
        k = np.zeros(1, dtype=np.int32)
        lib().orc_get_ncm_targets(self._h, _ptr(out), _ptr(k))
        return out[:int(k[0])]
