"""Thin Python binding of ``libhpclust.so`` (the C ABI in include/hpclust.h).

Argument marshalling only: every step runs in the CUDA kernels behind the C
ABI.  Tensors are torch CUDA tensors (PyTorch provides device memory and
streams); pointers, sizes and the current stream are passed through ctypes.
There is no CPU fallback: loading fails loudly when the library is missing
and cannot be built, and every call raises on a non-zero status.
"""
from __future__ import annotations

import ctypes
import math
from pathlib import Path

import torch

from . import _build

HPC_OK = 0
HPC_ERR_ARG = -1
HPC_ERR_NOMEM = -2
HPC_ERR_CUDA = -3
HPC_ERR_TIMEOUT = -4
HPC_ERR_NONFINITE = -5
HPC_ERR_DEGENERATE_ALL = -6
HPC_ERR_UNSUPPORTED = -7
HPC_FP32, HPC_BF16, HPC_FP8 = 0, 1, 2
HPC_COMPETITIVE, HPC_COOPERATIVE, HPC_HYBRID = 0, 1, 2
HPC_SEARCH_SIMT, HPC_SEARCH_SPLIT_TF32, HPC_SEARCH_TF32, HPC_SEARCH_SPLIT_BF16 = 0, 1, 2, 3
SEARCH_NAMES = {HPC_SEARCH_SIMT: "simt", HPC_SEARCH_SPLIT_TF32: "split_tf32",
                HPC_SEARCH_TF32: "tf32", HPC_SEARCH_SPLIT_BF16: "split_bf16"}
NFORMS = 4
(HPC_PROBE_FFMA, HPC_PROBE_FFMA2, HPC_PROBE_DFMA, HPC_PROBE_FMIN, HPC_PROBE_L2_READ,
 HPC_PROBE_HBM_READ) = range(6)
PROBES = {HPC_PROBE_FFMA: ("fp32 fma", "FMA/s"), HPC_PROBE_FFMA2: ("fp32x2 fma", "FMA/s"),
          HPC_PROBE_DFMA: ("fp64 fma", "FMA/s"), HPC_PROBE_FMIN: ("fp32 min", "op/s"),
          HPC_PROBE_L2_READ: ("L2 read", "B/s"), HPC_PROBE_HBM_READ: ("HBM read", "B/s")}

# Cost model of the objective's search forms (include/hpclust.h).
HPC_CM_NFEAT, HPC_CM_HIDDEN, HPC_CM_NPARAM = 8, 32, 1377

# The paper's hyperparameters (Section 6.5).
MAX_ITER = 300
REL_TOL = 1e-4
N_CANDIDATES = 3

_STATUS_NAMES = {v: k for k, v in dict(
    HPC_ERR_ARG=HPC_ERR_ARG, HPC_ERR_NOMEM=HPC_ERR_NOMEM, HPC_ERR_CUDA=HPC_ERR_CUDA,
    HPC_ERR_TIMEOUT=HPC_ERR_TIMEOUT, HPC_ERR_NONFINITE=HPC_ERR_NONFINITE,
    HPC_ERR_DEGENERATE_ALL=HPC_ERR_DEGENERATE_ALL,
    HPC_ERR_UNSUPPORTED=HPC_ERR_UNSUPPORTED).items()}


class HPCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class hpc_batch(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int32), ("s", ctypes.c_void_p), ("k", ctypes.c_void_p),
                ("group", ctypes.c_void_p), ("C_off", ctypes.c_void_p),
                ("K_off", ctypes.c_void_p), ("C", ctypes.c_void_p),
                ("degenerate", ctypes.c_void_p), ("fhat", ctypes.c_void_p),
                ("f_new", ctypes.c_void_p), ("iters", ctypes.c_void_p),
                ("accepted", ctypes.c_void_p), ("n_competitive", ctypes.c_int32),
                ("worker0", ctypes.c_int32), ("t_done", ctypes.c_void_p)]


_lib = None


def library_path() -> Path:
    return _build.OUT


def load() -> ctypes.CDLL:
    """Loads (building in-tree first if needed) the CUDA library."""
    global _lib
    if _lib is not None:
        return _lib
    if _build.stale():
        _build.build()
    L = ctypes.CDLL(str(_build.OUT))
    P, i32, i64, u32, u64, f64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                  ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double)
    sig = {
        "hpc_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, P], ctypes.c_int),
        "hpc_destroy": ([P], ctypes.c_int),
        "hpc_set_stream": ([P, P], ctypes.c_int),
        "hpc_sync_status": ([P], ctypes.c_int),
        "hpc_last_error": ([P], ctypes.c_char_p),
        "hpc_launch_count": ([P], i64),
        "hpc_reserve": ([P, i64], ctypes.c_int),
        "hpc_draw_sample": ([P, P, i64, i32, u64, u32, u32, i64, P, P], ctypes.c_int),
        "hpc_kmeanspp": ([P, P, i64, i32, i32, P, P, i32, u64, u32, u32], ctypes.c_int),
        "hpc_lloyd": ([P, P, i64, i32, i32, P, P, i32, f64, i32, P, P, P], ctypes.c_int),
        "hpc_objective": ([P, P, i64, i32, P, i32, P, i32, P, P], ctypes.c_int),
        "hpc_selftest_wait_timeout": ([P, i64], ctypes.c_int),
        "hpc_set_tensor_cores": ([P, ctypes.c_int], ctypes.c_int),
        "hpc_round": ([P, P, i64, i32, ctypes.POINTER(hpc_batch), i32, u64, u32, i32, f64,
                       i32, i32], ctypes.c_int),
        "hpc_round_prepare": ([P, P, i64, i32, ctypes.POINTER(hpc_batch), i32, u64, u32, i32,
                               f64, i32, i32], ctypes.c_int),
        "hpc_round_enqueue": ([P], ctypes.c_int),
        "hpc_set_objective_form": ([P, i32, i32, i32], ctypes.c_int),
        "hpc_peak_probe": ([i32, i32, P, ctypes.POINTER(f64), ctypes.POINTER(f64)], ctypes.c_int),
        "hpc_objective_form": ([P, i64, i32, i32], ctypes.c_int),
        "hpc_lloyd_cta_plan": ([i32, P, P, P, i32, P, P, P, P, P], ctypes.c_int),
        "hpc_lloyd_schedule": ([P, i64, i32, i32, ctypes.POINTER(ctypes.c_int32), i32],
                               ctypes.c_int),
        "hpc_set_phase_timing": ([P, i32], ctypes.c_int),
        "hpc_timestamp": ([P, P], ctypes.c_int),
        "hpc_set_search_stats": ([P, i32], ctypes.c_int),
        "hpc_search_stats": ([P, ctypes.POINTER(ctypes.c_int64), i32], ctypes.c_int),
        "hpc_phase_times": ([P, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "hpc_autotune_objective": ([P, P, i64, i32, P, i32, P, i32,
                                    ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "hpc_costmodel_loss_grad": ([P, P, P, P, i32, P, P], ctypes.c_int),
        "hpc_costmodel_train": ([P, P, P, P, P, P, i32, i32, i32, ctypes.c_float, P],
                                ctypes.c_int),
        "hpc_costmodel_predict": ([P, P, P, i32, P], ctypes.c_int),
        "hpc_costmodel_plan": ([ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32),
                                ctypes.c_float, ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "hpc_costmodel_features": ([P, P, P, i32, i32, ctypes.POINTER(ctypes.c_float),
                                    ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "hpc_autotune_objective_guided": ([P, P, i64, i32, P, i32, P, i32, P, ctypes.c_float,
                                           ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_float),
                                           ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "hpc_batch_save": ([P, ctypes.POINTER(hpc_batch), i32, u32, u64, i32, P, i64,
                            ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "hpc_batch_load": ([P, ctypes.POINTER(hpc_batch), i32, P, i64,
                            ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64),
                            ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need(t, dtype, name, device):
    if t is None:
        return
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if t.device != device:
        raise ValueError(f"{name}: expected a tensor on {device}, got {t.device}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")


class Context:
    """An ``hpc_ctx`` bound to one CUDA device and (by default) torch's
    current stream on that device."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self.lib = load()
        self.device = torch.device("cuda", device)
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.stream = st
        h = ctypes.c_void_p()
        rc = self.lib.hpc_create(ctypes.byref(h), device, ctypes.c_void_p(st.cuda_stream))
        if rc != HPC_OK:
            raise HPCError(rc, "hpc_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.hpc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        self._check(self.lib.hpc_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)))

    def _check(self, rc: int):
        if rc != HPC_OK:
            raise HPCError(rc, self.lib.hpc_last_error(self.h).decode())

    def sync_status(self) -> int:
        return int(self.lib.hpc_sync_status(self.h))

    def check_status(self):
        """Synchronise and raise if a device-side error was recorded."""
        self._check(self.sync_status())

    def launch_count(self) -> int:
        return int(self.lib.hpc_launch_count(self.h))

    def reserve(self, nbytes: int):
        self._check(self.lib.hpc_reserve(self.h, int(nbytes)))

    def set_tensor_cores(self, mode):
        """Tensor-core search: False/0 never, True/1 wherever built, 2 auto
        (the default; see include/hpclust.h)."""
        self._check(self.lib.hpc_set_tensor_cores(self.h, int(mode)))

    def set_objective_form(self, d: int, k: int, form: int):
        """Search form of hpc_objective for shape (d, k) in mode 2 (-1 clears)."""
        self._check(self.lib.hpc_set_objective_form(self.h, int(d), int(k), int(form)))

    def objective_form(self, n: int, d: int, k: int) -> int:
        rc = int(self.lib.hpc_objective_form(self.h, int(n), int(d), int(k)))
        if rc < 0:
            self._check(rc)
        return rc

    def lloyd_schedule(self, s: int, d: int, k: int) -> dict:
        """The launch hpc_lloyd would make for one sample of s rows (see
        hpc_lloyd_schedule in include/hpclust.h)."""
        out = (ctypes.c_int32 * 5)()
        self._check(self.lib.hpc_lloyd_schedule(self.h, int(s), int(d), int(k), out, 5))
        return {"blocks": int(out[0]), "smem_sums": bool(out[1]), "xstage": bool(out[2]),
                "smem_bytes": int(out[3]), "form": SEARCH_NAMES.get(int(out[4]), int(out[4]))}

    def set_search_stats(self, on: bool):
        """Count the stages of the split-BF16 tensor-core search."""
        self._check(self.lib.hpc_set_search_stats(self.h, int(bool(on))))

    def search_stats(self, reset: bool = False) -> dict:
        """Rows through each stage of the split-BF16 search since the last reset."""
        out = (ctypes.c_int64 * 4)()
        self._check(self.lib.hpc_search_stats(self.h, out, int(bool(reset))))
        return {"rows": int(out[0]), "near": int(out[1]), "all_centroids": int(out[2]),
                "fp64": int(out[3])}

    def timestamp(self, out=None):
        """A device int64 tensor that receives the device time (ns) once the
        work queued before it has run."""
        if out is None:
            out = torch.zeros(1, dtype=torch.int64, device=self.device)
        self._check(self.lib.hpc_timestamp(self.h, _ptr(out)))
        return out

    def set_phase_timing(self, on: bool):
        """Record CUDA events around every launch of later rounds."""
        self._check(self.lib.hpc_set_phase_timing(self.h, int(bool(on))))

    def phase_times(self) -> dict:
        """Milliseconds of the latest timed round per phase."""
        ms = (ctypes.c_float * 3)()
        self._check(self.lib.hpc_phase_times(self.h, ms))
        return {"sample": float(ms[0]), "kmeanspp": float(ms[1]), "lloyd": float(ms[2])}

    def autotune_objective(self, X, C, degenerate=None, reps: int = 5):
        """Times every search form built for C's shape on rows X, keeps the
        fastest for (d, k); returns (form, {form name: ms per call})."""
        n, d = X.shape
        k = C.shape[0]
        _need(X, torch.float32, "X", self.device)
        _need(C, torch.float32, "C", self.device)
        _need(degenerate, torch.uint8, "degenerate", self.device)
        form = ctypes.c_int32(-1)
        ms = (ctypes.c_float * NFORMS)()
        self._check(self.lib.hpc_autotune_objective(self.h, _ptr(X), n, d, _ptr(C), k,
                                                    _ptr(degenerate), int(reps),
                                                    ctypes.byref(form), ms))
        return int(form.value), {SEARCH_NAMES[i]: float(ms[i]) for i in range(NFORMS)
                                 if ms[i] >= 0}

    def autotune_objective_guided(self, X, C, params, degenerate=None, reps: int = 5,
                                  margin: float = 0.25):
        """hpc_autotune_objective guided by the cost-model network `params`:
        returns (form, {form name: ms per call of each timed form}, forms timed)."""
        n, d = X.shape
        k = C.shape[0]
        _need(X, torch.float32, "X", self.device)
        _need(C, torch.float32, "C", self.device)
        _need(params, torch.float32, "params", self.device)
        _need(degenerate, torch.uint8, "degenerate", self.device)
        form = ctypes.c_int32(-1)
        timed = ctypes.c_int32(0)
        ms = (ctypes.c_float * NFORMS)()
        self._check(self.lib.hpc_autotune_objective_guided(
            self.h, _ptr(X), n, d, _ptr(C), k, _ptr(degenerate), int(reps), _ptr(params),
            float(margin), ctypes.byref(form), ms, ctypes.byref(timed)))
        return (int(form.value),
                {SEARCH_NAMES[i]: float(ms[i]) for i in range(NFORMS) if ms[i] >= 0},
                int(timed.value))

    def selftest_wait_timeout(self, limit_ns: int):
        """Launches the bounded-wait self-test (see include/hpclust.h)."""
        self._check(self.lib.hpc_selftest_wait_timeout(self.h, int(limit_ns)))


def hpc_draw_sample(ctx: Context, X, seed: int, worker: int, round_: int, s: int,
                    S_out=None, idx_out=None):
    n, d = X.shape
    _need(X, torch.float32, "X", ctx.device)
    if S_out is None:
        S_out = torch.empty((s, d), dtype=torch.float32, device=ctx.device)
    _need(S_out, torch.float32, "S_out", ctx.device)
    _need(idx_out, torch.int64, "idx_out", ctx.device)
    ctx._check(ctx.lib.hpc_draw_sample(ctx.h, _ptr(X), n, d, seed, worker, round_, s,
                                       _ptr(S_out), _ptr(idx_out)))
    return S_out, idx_out


def hpc_kmeanspp(ctx: Context, S, C, degenerate=None, n_candidates: int = N_CANDIDATES,
                 seed: int = 0, worker: int = 0, round_: int = 0):
    """Seeds (in place) the degenerate rows of C; returns (C, degenerate)."""
    s, d = S.shape
    k = C.shape[0]
    _need(S, torch.float32, "S", ctx.device)
    _need(C, torch.float32, "C", ctx.device)
    _need(degenerate, torch.uint8, "degenerate", ctx.device)
    ctx._check(ctx.lib.hpc_kmeanspp(ctx.h, _ptr(S), s, d, k, _ptr(C), _ptr(degenerate),
                                    n_candidates, seed, worker, round_))
    return C, degenerate


def hpc_lloyd(ctx: Context, S, C, degenerate=None, max_iter: int = MAX_ITER,
              rel_tol: float = REL_TOL, prec: int = HPC_FP32, labels_out=None,
              f_out=None, iters_out=None):
    """Runs Lloyd in place on C / degenerate; returns (f_out, iters_out) device tensors."""
    s, d = S.shape
    k = C.shape[0]
    _need(S, torch.float32, "S", ctx.device)
    _need(C, torch.float32, "C", ctx.device)
    _need(degenerate, torch.uint8, "degenerate", ctx.device)
    _need(labels_out, torch.int32, "labels_out", ctx.device)
    if f_out is None:
        f_out = torch.empty(1, dtype=torch.float64, device=ctx.device)
    if iters_out is None:
        iters_out = torch.empty(1, dtype=torch.int32, device=ctx.device)
    ctx._check(ctx.lib.hpc_lloyd(ctx.h, _ptr(S), s, d, k, _ptr(C), _ptr(degenerate), max_iter,
                                 rel_tol, prec, _ptr(labels_out), _ptr(f_out), _ptr(iters_out)))
    return f_out, iters_out


def hpc_objective(ctx: Context, X, C, degenerate=None, prec: int = HPC_FP32, f_out=None,
                  labels_out=None):
    n, d = X.shape
    k = C.shape[0]
    _need(X, torch.float32, "X", ctx.device)
    _need(C, torch.float32, "C", ctx.device)
    _need(degenerate, torch.uint8, "degenerate", ctx.device)
    _need(labels_out, torch.int32, "labels_out", ctx.device)
    if f_out is None:
        f_out = torch.empty(1, dtype=torch.float64, device=ctx.device)
    ctx._check(ctx.lib.hpc_objective(ctx.h, _ptr(X) if n > 0 else None, n, d, _ptr(C), k,
                                     _ptr(degenerate), prec, _ptr(f_out), _ptr(labels_out)))
    return f_out


class Batch:
    """Worker set for hpc_round: host descriptors plus device state."""

    def __init__(self, d: int, s, k, group=None, device=None, n_competitive: int = 0,
                 worker0: int = 0):
        import numpy as np
        self.d = d
        self.n_competitive = int(n_competitive)  # HPC_HYBRID: rounds of the competitive phase
        self.worker0 = int(worker0)  # global index of worker 0 (its random streams)
        self.device = device or torch.device("cuda", 0)
        self.s = np.ascontiguousarray(s, dtype=np.int64)
        self.k = np.ascontiguousarray(k, dtype=np.int32)
        self.W = len(self.s)
        self.group = (np.zeros(self.W, np.int32) if group is None
                      else np.ascontiguousarray(group, dtype=np.int32))
        self.C_off = np.zeros(self.W, np.int64)
        self.K_off = np.zeros(self.W, np.int64)
        nf = nk = 0
        for w in range(self.W):
            self.C_off[w] = nf
            self.K_off[w] = nk
            nf += int(self.k[w]) * d
            nf = (nf + 3) // 4 * 4      # keep every worker's centroids 16-byte aligned
            nk += int(self.k[w])
        self.C = torch.zeros(nf, dtype=torch.float32, device=self.device)
        self.degenerate = torch.ones(nk, dtype=torch.uint8, device=self.device)
        self.fhat = torch.full((self.W,), math.inf, dtype=torch.float64, device=self.device)
        self.f_new = torch.zeros(self.W, dtype=torch.float64, device=self.device)
        self.iters = torch.zeros(self.W, dtype=torch.int32, device=self.device)
        self.accepted = torch.zeros(self.W, dtype=torch.uint8, device=self.device)
        # per round, the device time each worker's run ended (hpc_timestamp's clock)
        self.t_done = torch.zeros(self.W, dtype=torch.int64, device=self.device)

    def struct(self) -> hpc_batch:
        return hpc_batch(self.W, self.s.ctypes.data, self.k.ctypes.data, self.group.ctypes.data,
                         self.C_off.ctypes.data, self.K_off.ctypes.data, self.C.data_ptr(),
                         self.degenerate.data_ptr(), self.fhat.data_ptr(), self.f_new.data_ptr(),
                         self.iters.data_ptr(), self.accepted.data_ptr(), self.n_competitive,
                         self.worker0, self.t_done.data_ptr())

    def save(self, ctx: "Context", path, next_round: int, seed: int, strategy: int):
        """Writes the checkpoint of hpc_batch_save to the file `path`."""
        Path(path).write_bytes(hpc_batch_save(ctx, self, next_round, seed, strategy))

    def load(self, ctx: "Context", path):
        """Restores the state saved by save(); returns (next_round, seed, strategy)."""
        return hpc_batch_load(ctx, self, Path(path).read_bytes())

    def centroids(self, w: int):
        k = int(self.k[w])
        o = int(self.C_off[w])
        return (self.C[o: o + k * self.d].view(k, self.d),
                self.degenerate[int(self.K_off[w]): int(self.K_off[w]) + k])


def hpc_round(ctx: Context, X, batch: Batch, strategy: int, seed: int, round_: int,
              max_iter: int = MAX_ITER, rel_tol: float = REL_TOL,
              n_candidates: int = N_CANDIDATES, prec: int = HPC_FP32):
    n, d = X.shape
    _need(X, torch.float32, "X", ctx.device)
    b = batch.struct()
    ctx._check(ctx.lib.hpc_round(ctx.h, _ptr(X), n, d, ctypes.byref(b), strategy, seed, round_,
                                 max_iter, rel_tol, n_candidates, prec))


def hpc_round_prepare(ctx: Context, X, batch: Batch, strategy: int, seed: int, round0: int = 0,
                      max_iter: int = MAX_ITER, rel_tol: float = REL_TOL,
                      n_candidates: int = N_CANDIDATES, prec: int = HPC_FP32):
    """Set-up of a round that hpc_round_enqueue then enqueues (and a stream
    capture can record) round after round."""
    n, d = X.shape
    _need(X, torch.float32, "X", ctx.device)
    b = batch.struct()
    ctx._check(ctx.lib.hpc_round_prepare(ctx.h, _ptr(X), n, d, ctypes.byref(b), strategy, seed,
                                         round0, max_iter, rel_tol, n_candidates, prec))


def hpc_round_enqueue(ctx: Context):
    ctx._check(ctx.lib.hpc_round_enqueue(ctx.h))


def hpc_batch_save(ctx: Context, batch: Batch, next_round: int, seed: int, strategy: int) -> bytes:
    """The batch's incumbents, flags and fhat with the next round, seed and
    strategy, as the bytes of the checkpoint format in include/hpclust.h."""
    b = batch.struct()
    need = ctypes.c_int64(0)
    ctx._check(ctx.lib.hpc_batch_save(ctx.h, ctypes.byref(b), batch.d, next_round, seed, strategy,
                                      None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(int(need.value))
    ctx._check(ctx.lib.hpc_batch_save(ctx.h, ctypes.byref(b), batch.d, next_round, seed, strategy,
                                      buf, need.value, ctypes.byref(need)))
    return buf.raw


def hpc_batch_load(ctx: Context, batch: Batch, blob: bytes):
    """Writes a checkpoint back into the batch; returns (next_round, seed, strategy)."""
    b = batch.struct()
    buf = ctypes.create_string_buffer(bytes(blob), len(blob))
    r, sd, st = ctypes.c_uint32(0), ctypes.c_uint64(0), ctypes.c_int32(0)
    ctx._check(ctx.lib.hpc_batch_load(ctx.h, ctypes.byref(b), batch.d, buf, len(blob),
                                      ctypes.byref(r), ctypes.byref(sd), ctypes.byref(st)))
    return int(r.value), int(sd.value), int(st.value)


def hpc_peak_probe(kind: int, device: int = 0, stream: torch.cuda.Stream | None = None):
    """Measured rate of one throughput probe (include/hpclust.h); returns
    (rate, ms per launch)."""
    lib = load()
    st = stream if stream is not None else torch.cuda.current_stream(torch.device("cuda", device))
    rate, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = lib.hpc_peak_probe(int(kind), int(device), ctypes.c_void_p(st.cuda_stream),
                            ctypes.byref(rate), ctypes.byref(ms))
    if rc != HPC_OK:
        raise HPCError(rc, "hpc_peak_probe failed")
    return float(rate.value), float(ms.value)


# ---- cost model of the objective's search forms -------------------------

def _cm_check(params, feats, N, dev):
    _need(params, torch.float32, "params", dev)
    _need(feats, torch.float32, "feats", dev)
    if params.numel() != HPC_CM_NPARAM:
        raise ValueError(f"params: expected {HPC_CM_NPARAM} values")
    if feats.numel() != N * HPC_CM_NFEAT:
        raise ValueError(f"feats: expected {N} x {HPC_CM_NFEAT} values")


def hpc_costmodel_loss_grad(ctx: Context, params, feats, targets):
    """(loss, gradient) device tensors of the network's mean squared error."""
    N = targets.numel()
    _cm_check(params, feats, N, ctx.device)
    _need(targets, torch.float32, "targets", ctx.device)
    loss = torch.empty(1, dtype=torch.float32, device=ctx.device)
    grad = torch.empty(HPC_CM_NPARAM, dtype=torch.float32, device=ctx.device)
    ctx._check(ctx.lib.hpc_costmodel_loss_grad(ctx.h, _ptr(params), _ptr(feats), _ptr(targets),
                                               N, _ptr(loss), _ptr(grad)))
    return loss, grad


def hpc_costmodel_train(ctx: Context, params, m, v, feats, targets, steps: int, step0: int = 0,
                        lr: float = 3e-3, loss_out=None):
    """`steps` Adam steps on params (in place), moments m, v carried."""
    N = targets.numel()
    _cm_check(params, feats, N, ctx.device)
    for t, name in ((m, "m"), (v, "v"), (targets, "targets"), (loss_out, "loss_out")):
        _need(t, torch.float32, name, ctx.device)
    if m.numel() != HPC_CM_NPARAM or v.numel() != HPC_CM_NPARAM:
        raise ValueError("m, v: one value per parameter")
    if loss_out is not None and loss_out.numel() < steps:
        raise ValueError("loss_out: one value per step")
    ctx._check(ctx.lib.hpc_costmodel_train(ctx.h, _ptr(params), _ptr(m), _ptr(v), _ptr(feats),
                                           _ptr(targets), N, int(steps), int(step0), float(lr),
                                           _ptr(loss_out)))


def hpc_costmodel_predict(ctx: Context, params, feats):
    N = feats.numel() // HPC_CM_NFEAT
    _cm_check(params, feats, N, ctx.device)
    out = torch.empty(N, dtype=torch.float32, device=ctx.device)
    ctx._check(ctx.lib.hpc_costmodel_predict(ctx.h, _ptr(params), _ptr(feats), N, _ptr(out)))
    return out


def hpc_costmodel_features(ctx: Context, C, degenerate=None):
    """(3 x HPC_CM_NFEAT host float tensor, [supported per form])."""
    k, d = C.shape
    _need(C, torch.float32, "C", ctx.device)
    _need(degenerate, torch.uint8, "degenerate", ctx.device)
    feats = (ctypes.c_float * (3 * HPC_CM_NFEAT))()
    sup = (ctypes.c_int32 * 3)()
    ctx._check(ctx.lib.hpc_costmodel_features(ctx.h, _ptr(C), _ptr(degenerate), d, k, feats,
                                              sup))
    return (torch.tensor(list(feats), dtype=torch.float32).view(3, HPC_CM_NFEAT),
            [int(x) for x in sup])


def hpc_costmodel_plan(pred, supported, margin: float):
    """The guided search's plan (host only): (forms ranked by predicted time,
    1 where that form is timed), each of length 3 with -1 / 0 past the built
    forms."""
    p = (ctypes.c_float * 3)(*[float(x) for x in pred])
    sp = (ctypes.c_int32 * 3)(*[int(x) for x in supported])
    order = (ctypes.c_int32 * 3)()
    timed = (ctypes.c_int32 * 3)()
    rc = int(load().hpc_costmodel_plan(p, sp, float(margin), order, timed))
    if rc < 0:
        raise HPCError(rc, "hpc_costmodel_plan: bad arguments")
    return list(order), list(timed)


def lloyd_cta_plan(s, k, u, ctas: int) -> dict:
    """The CTA plan of a batched split-BF16 Lloyd launch (host only; see
    hpc_lloyd_cta_plan in include/hpclust.h): the first worker of each
    CTA's set (-2: none, it takes from the list), the list, the worker each
    set runs after each worker (-1: none), and each worker's CTAs."""
    import numpy as np
    L = load()
    s = np.ascontiguousarray(s, dtype=np.int64)
    k = np.ascontiguousarray(k, dtype=np.int32)
    u = np.ascontiguousarray(u, dtype=np.int32)
    W = len(s)
    cta_task = np.empty(max(int(ctas), 1), np.int32)
    lst = np.empty(max(W, 1), np.int32)
    nb = np.empty(max(W, 1), np.int32)
    nxt = np.empty(max(W, 1), np.int32)
    nlist = ctypes.c_int32(0)
    rc = L.hpc_lloyd_cta_plan(W, s.ctypes.data, k.ctypes.data, u.ctypes.data, int(ctas),
                              cta_task.ctypes.data, lst.ctypes.data, ctypes.addressof(nlist),
                              nxt.ctypes.data, nb.ctypes.data)
    if rc != 0:
        raise HPCError(rc, "hpc_lloyd_cta_plan")
    return {"cta_task": cta_task[:int(ctas)], "list": lst[:nlist.value], "next": nxt[:W],
            "nblocks": nb[:W]}

