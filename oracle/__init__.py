"""HPClust CPU oracle (double precision, plain loops).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The GPU library and its Python
binding never import it, and it shares no code with them.

Every function follows a passage of arXiv 2311.04517 (HPClust); the C source
``hpclust_oracle.c`` cites the passage beside each step.  Parity pins live in
``tests/test_oracle_pins.py``; every function below has at least one pin that
does not go through the oracle itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "hpclust_oracle.c"
_LIB = _HERE / "liboracle.so"

OK = 0
ERR_ARG = -1
ERR_NOMEM = -2
ERR_DEGENERATE_ALL = -6
COMPETITIVE = 0
COOPERATIVE = 1
HYBRID = 2
TAG_SAMPLE = 0
TAG_SEED = 1


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (OpenMP, no floating-point contraction)."""
    if not force and _LIB.exists() and _LIB.stat().st_mtime >= _SRC.stat().st_mtime:
        return _LIB
    tmp = _LIB.with_suffix(f".{os.getpid()}.tmp.so")
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-std=c11", "-shared", "-fPIC", str(_SRC), "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_LIB))
        P = ctypes.c_void_p
        i64, i32, u64, u32, f64 = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                   ctypes.c_uint32, ctypes.c_double)
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_philox4x64_10.argtypes = [P, P, P]
        L.orc_philox4x64_10.restype = None
        L.orc_draw.argtypes = [u64, u32, u32, u32, u64]
        L.orc_draw.restype = u64
        L.orc_draw_sample.argtypes = [P, i64, i32, u64, u32, u32, i64, P, P]
        L.orc_draw_sample.restype = ctypes.c_int
        L.orc_dist32.argtypes = [P, P, i32]
        L.orc_dist32.restype = ctypes.c_float
        L.orc_assign.argtypes = [P, i64, i32, P, i32, P, P, P, P]
        L.orc_assign.restype = f64
        L.orc_update.argtypes = [P, i64, i32, P, i32, P, P]
        L.orc_update.restype = ctypes.c_int
        L.orc_lloyd.argtypes = [P, i64, i32, i32, P, P, i32, f64, P, P, P, P]
        L.orc_lloyd.restype = ctypes.c_int
        L.orc_fixed_scale.argtypes = [ctypes.c_float, i64]
        L.orc_fixed_scale.restype = ctypes.c_int
        L.orc_quant.argtypes = [ctypes.c_float, ctypes.c_int]
        L.orc_quant.restype = i64
        L.orc_d2_pick.argtypes = [P, i64, u64]
        L.orc_d2_pick.restype = i64
        L.orc_kmeanspp.argtypes = [P, i64, i32, i32, P, P, i32, u64, u32, u32, P, P]
        L.orc_kmeanspp.restype = ctypes.c_int
        L.orc_objective.argtypes = [P, i64, i32, P, i32, P, P]
        L.orc_objective.restype = f64
        L.orc_round.argtypes = [P, i64, i32, i32, P, P, P, P, P, P, P, P, i32, u64, u32,
                                i32, f64, i32, P, P, P, i32, i32]
        L.orc_round.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def philox4x64_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_p(c), _p(k), _p(out))
    return out


def draw(seed: int, worker: int, round_: int, tag: int, j: int) -> int:
    return int(lib().orc_draw(seed, worker, round_, tag, j))


def draw_sample(X, seed: int, worker: int, round_: int, s: int):
    X = _f32(X)
    n, d = X.shape
    S = np.empty((s, d), dtype=np.float32)
    idx = np.empty(s, dtype=np.int64)
    rc = lib().orc_draw_sample(_p(X), n, d, seed, worker, round_, s, _p(S), _p(idx))
    if rc:
        raise ValueError(f"orc_draw_sample failed: {rc}")
    return S, idx


def sample_indices(n: int, seed: int, worker: int, round_: int, s: int) -> np.ndarray:
    """The row indices draw_sample takes (Section 3's random sample, with
    replacement): index i is floor(r_i * n / 2^64) with r_i draw i of stream
    (seed, worker, round, tag 0).  For data too large to pass whole to
    draw_sample; the rows themselves are then X[indices]."""
    out = np.empty(s, dtype=np.int64)
    L = lib()
    for i in range(s):
        r = int(L.orc_draw(seed, worker, round_, TAG_SAMPLE, i))
        out[i] = (r * int(n)) >> 64
    return out


def dist32(x, c) -> float:
    x = _f32(x)
    c = _f32(c)
    return float(lib().orc_dist32(_p(x), _p(c), x.shape[-1]))


def assign(S, C, degenerate=None):
    """Returns (labels, d1, d2, f) in double precision."""
    S = _f32(S)
    C = _f32(C)
    s, d = S.shape
    k = C.shape[0]
    deg = None if degenerate is None else np.ascontiguousarray(degenerate, dtype=np.uint8)
    labels = np.empty(s, dtype=np.int32)
    d1 = np.empty(s, dtype=np.float64)
    d2 = np.empty(s, dtype=np.float64)
    f = lib().orc_assign(_p(S), s, d, _p(C), k, _p(deg), _p(labels), _p(d1), _p(d2))
    return labels, d1, d2, float(f)


def update(S, labels, C, degenerate):
    """Returns (C_new, degenerate_new); inputs are not modified."""
    S = _f32(S)
    C = _f32(C).copy()
    deg = np.ascontiguousarray(degenerate, dtype=np.uint8).copy()
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    s, d = S.shape
    rc = lib().orc_update(_p(S), s, d, _p(lab), C.shape[0], _p(C), _p(deg))
    if rc:
        raise ValueError(f"orc_update failed: {rc}")
    return C, deg


def lloyd(S, C0, degenerate=None, max_iter: int = 300, rel_tol: float = 1e-4):
    """Returns dict(C, degenerate, labels, f, iters, f_trace, rc)."""
    S = _f32(S)
    C = _f32(C0).copy()
    s, d = S.shape
    k = C.shape[0]
    deg = (np.zeros(k, np.uint8) if degenerate is None
           else np.ascontiguousarray(degenerate, dtype=np.uint8).copy())
    labels = np.empty(s, dtype=np.int32)
    f = ctypes.c_double(0.0)
    it = ctypes.c_int32(0)
    trace = np.full(max_iter + 1, np.nan)
    rc = lib().orc_lloyd(_p(S), s, d, k, _p(C), _p(deg), max_iter, rel_tol, _p(labels),
                         ctypes.byref(f), ctypes.byref(it), _p(trace))
    return dict(C=C, degenerate=deg, labels=labels, f=f.value, iters=it.value,
                f_trace=trace[: it.value + 1], rc=rc)


def fixed_scale(M: float, s: int) -> int:
    return int(lib().orc_fixed_scale(M, s))


def quant(w: float, F: int) -> int:
    return int(lib().orc_quant(w, F))


def d2_pick(w, r: int) -> int:
    w = _f32(w)
    return int(lib().orc_d2_pick(_p(w), w.shape[0], r))


def kmeanspp(S, C0, degenerate, L: int = 3, seed: int = 0, worker: int = 0, round_: int = 0):
    """Returns dict(C, degenerate, cand, phi, rc)."""
    S = _f32(S)
    C = _f32(C0).copy()
    s, d = S.shape
    k = C.shape[0]
    deg = np.ascontiguousarray(degenerate, dtype=np.uint8).copy()
    cand = np.empty((k, L), dtype=np.int64)
    phi = np.empty((k, L), dtype=np.int64)
    rc = lib().orc_kmeanspp(_p(S), s, d, k, _p(C), _p(deg), L, seed, worker, round_,
                            _p(cand), _p(phi))
    return dict(C=C, degenerate=deg, cand=cand, phi=phi, rc=rc)


def objective(X, C, degenerate=None, want_labels: bool = False):
    X = _f32(X)
    C = _f32(C)
    n, d = X.shape
    deg = None if degenerate is None else np.ascontiguousarray(degenerate, dtype=np.uint8)
    labels = np.empty(n, dtype=np.int32) if want_labels else None
    f = float(lib().orc_objective(_p(X), n, d, _p(C), C.shape[0], _p(deg), _p(labels)))
    return (f, labels) if want_labels else f


class RoundState:
    """Per-worker incumbents for a round sequence (Algorithms 3-5 state)."""

    def __init__(self, d: int, s, k, group=None):
        self.d = d
        self.s = np.ascontiguousarray(s, dtype=np.int64)
        self.k = np.ascontiguousarray(k, dtype=np.int32)
        W = len(self.s)
        self.group = (np.zeros(W, np.int32) if group is None
                      else np.ascontiguousarray(group, dtype=np.int32))
        self.C_off = np.zeros(W, np.int64)
        self.K_off = np.zeros(W, np.int64)
        acc_f = acc_k = 0
        for w in range(W):
            self.C_off[w] = acc_f
            self.K_off[w] = acc_k
            acc_f += int(self.k[w]) * d
            acc_k += int(self.k[w])
        self.C_pool = np.zeros(acc_f, np.float32)
        self.deg_pool = np.ones(acc_k, np.uint8)       # all centroids start degenerate
        self.fhat = np.full(W, np.inf)                  # incumbent objective per point

    def centroids(self, w: int):
        k = int(self.k[w])
        C = self.C_pool[self.C_off[w]: self.C_off[w] + k * self.d].reshape(k, self.d)
        deg = self.deg_pool[self.K_off[w]: self.K_off[w] + k]
        return C.copy(), deg.copy()


def round_(X, state: RoundState, strategy: int, seed: int, round_idx: int,
           max_iter: int = 300, rel_tol: float = 1e-4, L: int = 3, n_competitive: int = 0,
           worker0: int = 0):
    """Runs one round in place on ``state``; returns dict(f_new, iters, accepted).

    strategy HYBRID (Algorithm 5): round_idx < n_competitive runs the
    competitive phase, later rounds the cooperative one.  worker0: the
    global index of the state's first worker (its random streams)."""
    X = _f32(X)
    n, d = X.shape
    W = len(state.s)
    f_new = np.zeros(W)
    iters = np.zeros(W, np.int32)
    acc = np.zeros(W, np.uint8)
    rc = lib().orc_round(_p(X), n, d, W, _p(state.s), _p(state.k), _p(state.group),
                         _p(state.C_pool), _p(state.C_off), _p(state.deg_pool),
                         _p(state.K_off), _p(state.fhat), strategy, seed, round_idx,
                         max_iter, rel_tol, L, _p(f_new), _p(iters), _p(acc), n_competitive,
                         int(worker0))
    if rc:
        raise ValueError(f"orc_round failed: {rc}")
    return dict(f_new=f_new, iters=iters, accepted=acc.astype(bool))
