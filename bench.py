#!/usr/bin/env python3
"""Throughput of the HPClust hot path on GB300: point-centroid distances/s.

One step = one HPClust round on the benchmark workload (sample draw,
K-means++ reseeding of degenerate centroids, Lloyd to the Section 6.5 stop
rule, incumbent test), replayed from a CUDA graph that recorded one round
(--no-graph: issued call by call), followed by the full-data objective of
the best incumbent of each sharing group (Eq. 1 over all n rows).  Distances
counted per step: (Lloyd assignments) x s x k + n x k.  Default workload:
"large", the largest configuration that fits one GPU (n = 2 x 10^8 points in
64 dims, 500 Gaussians with Zipf(1.1) weights, 51 GB; 128 workers with
k = 500 and samples of 65,536 to 1,048,576 rows).

Prints one JSON line (rank 0).  Arms:
  --impl mine       the CUDA library (default)
  --impl reference  the CPU oracle as the reference arm (host cores)
Multi-GPU (torchrun): one job over the ranks -- workers split into contiguous
ranges, the objective's rows into blocks (paper_2311_04517_gb300/multirank.py);
barrier and max-over-ranks timing, the work summed over the ranks.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import re
import statistics
import sys
import threading
import time
from dataclasses import replace
from pathlib import Path

ROOT = Path(__file__).resolve().parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_2311_04517_gb300 import synth  # noqa: E402

METRIC = "point-centroid distances/s"
UNIT = "distances/s"
FALLBACK_HBM = 6800.0
FALLBACK_BF16_SUSTAINED = 1700.0   # TFLOP/s, the profiling recipe's sustained fallback
TIMED_BUDGET_S = 45.0              # timed work of a default run


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None,
                   help="timed steps (default: about TIMED_BUDGET_S of timed work, at least 5 "
                        "and at most 100, from the last warm-up step; 5 for --impl reference)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["mine", "reference"], default="mine")
    p.add_argument("--workload", default="large")
    p.add_argument("--workers", type=int, default=None,
                   help="a smaller case of the workload: its first this many workers "
                        "(for profiler captures; not a bench configuration)")
    p.add_argument("--strategy", choices=["competitive", "cooperative", "hybrid"],
                   default="competitive")
    p.add_argument("--n-competitive", type=int, default=None,
                   help="hybrid: rounds of the competitive phase (default: half the run)")
    p.add_argument("--no-graph", dest="graph", action="store_false",
                   help="issue every round with hpc_round instead of replaying one round "
                        "recorded in a CUDA graph (hpc_round_prepare / hpc_round_enqueue)")
    p.add_argument("--tensor-cores", type=int, choices=[0, 1, 2], default=2,
                   help="objective search: 0 CUDA cores, 1 tensor cores wherever built, 2 auto")
    p.add_argument("--rows", type=int, default=None,
                   help="a smaller case of the workload: this many data rows instead of n "
                        "(for profiler captures; not a bench configuration)")
    p.add_argument("--no-autotune", dest="autotune", action="store_false",
                   help="keep the built-in objective search forms instead of timing every "
                        "form on the workload before the timed steps (hpc_autotune_objective)")
    p.add_argument("--tto-rounds", type=int, default=None,
                   help="rounds of the time-to-objective comparison with the plain FP32 path "
                        "(default: the workload's rounds, at most 10; 0 skips it)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--scaling-experiment", action="store_true",
                   help="Section 6.8's scaling experiment on the GPU instead of the benchmark "
                        "step: m = 3^(i+7) points (i = 0..8), the three strategies, "
                        "--scaling-rounds rounds each")
    p.add_argument("--scaling-rounds", type=int, default=30)
    p.add_argument("--e2e-steps", type=int, default=None)
    return p.parse_args()


# The arithmetic roofline of the CUDA-core search: 152 SMs x 128 FP32 lanes,
# one fused multiply-add (2 flops) per lane per clock at the 2070 MHz
# maximum SM clock.
SMS, FP32_LANES_PER_SM, SM_MAX_MHZ = 152, 128, 2070.0
ALU_PEAK_TFLOPS = 2.0 * SMS * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12


# the tensor-core search forms: products per FP32 product and the dtype's
# share of the BF16 rate (NVIDIA's dense figures: TF32 1.1 of BF16's 2.25
# PFLOP/s); split forms emulate an FP32 product with three
TENSOR_FORMS = {"tf32": (1, 1.1 / 2.25), "split_tf32": (3, 1.1 / 2.25), "split_bf16": (3, 1.0)}


def tensor_peak(form: str):
    """(TFLOP/s of the form's FP32-equivalent products, source) from the
    measured sustained BF16 rate (the kernels run inside seconds-long steps)."""
    f = ROOT / "MEASURED_PEAKS.json"
    if f.exists():
        bf16, src = float(json.loads(f.read_text())["bf16_tflops_sustained"]), "measured"
    else:
        bf16, src = FALLBACK_BF16_SUSTAINED, "fallback"
    n, ratio = TENSOR_FORMS[form]
    return bf16 * ratio / n, (f"{src} bf16_tflops_sustained x {ratio:.3g} / {n} "
                              f"({n} {form.split('_')[-1]} product(s) per FP32 product)")


def roofline_bound(label: str, bytes_: float, flops: float, avg_ms: float, form: str,
                   hbm_gbs: float, hbm_src: str, traffic, extra=None):
    """Roofline of one kernel: HBM (bytes_ per launch) unless its
    contraction's flops take longer at the arithmetic peak than the bytes at
    the HBM peak.  The CUDA-core form (simt) is held against the FP32 FMA
    peak; the tensor-core forms against the tensor rate of their products
    (TENSOR_FORMS)."""
    t_hbm = bytes_ / (hbm_gbs * 1e9)
    if form == "simt":
        peak, peak_src, bound = (ALU_PEAK_TFLOPS,
                                 "152 SMs x 128 FP32 lanes x 2070 MHz, 2 flops per FMA", "alu")
    else:
        (peak, peak_src), bound = tensor_peak(form), "tensor"
    t_arith = flops / (peak * 1e12)
    entry = {"kernel": label, "traffic": traffic, "algorithmic_bytes_per_launch": bytes_,
             "algorithmic_flops_per_launch": flops, "avg_launch_ms": avg_ms, "form": form}
    if extra:
        entry.update(extra)
    if t_arith > t_hbm:
        achieved = flops / (avg_ms / 1e3) / 1e12
        entry.update({"bound": bound, "achieved": achieved, "peak": peak,
                      "peak_source": peak_src, "unit": "TFLOP/s", "frac": achieved / peak})
    else:
        achieved = bytes_ / (avg_ms / 1e3) / 1e9
        entry.update({"bound": "hbm", "achieved": achieved, "peak": hbm_gbs,
                      "peak_source": f"{hbm_src} hbm_gbs", "unit": "GB/s",
                      "frac": achieved / hbm_gbs})
    return entry


def roofline_entry(kernel: str, form: str, n: int, d: int, k_mean: float, avg_ms: float,
                   hbm_gbs: float, hbm_src: str, traffic):
    """The full-data objective's roofline: 4 n d bytes and 2 n k d flops per
    launch (k_mean the groups' mean k)."""
    return roofline_bound(f"{kernel} (full-data objective, Eq. 1)", float(n) * d * 4,
                          2.0 * n * k_mean * d, avg_ms, form, hbm_gbs, hbm_src, traffic)


def lloyd_roofline(kernel: str, form: str, passes_rows_k, d: int, launches: int, avg_ms: float,
                   hbm_gbs: float, hbm_src: str, traffic):
    """The Lloyd launch's roofline: each assignment pass of worker w reads
    its sample (4 s_w d bytes) and evaluates s_w k_w distances of 2 d flops
    (the x.c contraction); passes_rows_k = [(passes, s_w, k_w)] summed over
    the steps, divided over the launches."""
    rows = sum(float(p) * float(s_) for p, s_, _ in passes_rows_k)
    dists = sum(float(p) * float(s_) * float(k_) for p, s_, k_ in passes_rows_k)
    return roofline_bound(f"{kernel} (Lloyd iterations, Algorithm 1)", 4.0 * d * rows / launches,
                          2.0 * d * dists / launches, avg_ms, form, hbm_gbs, hbm_src, traffic,
                          {"launches_timed": launches})


def plan_balance(s, k, u_prev, u_now, ctas: int) -> dict:
    """The batched split-BF16 Lloyd's CTA plan as the device makes it from
    one step's update counts, timed with the next step's counts in units of
    distances (s k (u + 1) per worker): a set's CTAs run its workers one
    after another, each worker's work spread over them; a free CTA takes the
    next worker of the list (the earliest free first). Returns the plan's
    shape and its makespan over the balanced time (all work spread evenly
    over the CTAs); the kernel's time per distance is the launch's time over
    that makespan."""
    import heapq

    from paper_2311_04517_gb300 import hpclust as H
    s = np.asarray(s, np.int64)
    k = np.asarray(k, np.int64)
    plan = H.lloyd_cta_plan(s, k, np.asarray(u_prev, np.int32), int(ctas))
    work = s.astype(np.float64) * k * (np.clip(np.asarray(u_now, np.int64), 0, None) + 1)
    ct, nb, nxt = plan["cta_task"], plan["nblocks"], plan["next"]
    free = []
    for c, t in enumerate(ct):
        f = 0.0
        while t >= 0:
            f += float(work[t] / nb[t])
            t = int(nxt[t])
        free.append((f, c))
    heapq.heapify(free)
    for t in plan["list"]:
        f0, c = heapq.heappop(free)
        heapq.heappush(free, (f0 + float(work[t]), c))
    makespan = max(f for f, _ in free)
    return {"sets": len({int(t) for t in ct if t >= 0}), "set_ctas": int((ct >= 0).sum()),
            "list": int(len(plan["list"])),
            "makespan_over_balanced": float(makespan / (work.sum() / int(ctas)))}


def peaks():
    f = ROOT / "MEASURED_PEAKS.json"
    if f.exists():
        j = json.loads(f.read_text())
        return float(j["hbm_gbs"]), "measured"
    return FALLBACK_HBM, "fallback"


# the source files each profiled kernel is compiled from (its translation
# unit and the kernel headers it includes)
_COMMON = ["assign.cuh", "common.cuh", "kernels.h"]
KERNEL_SOURCES = {
    "objective_kernel": ["lloyd.cu"] + _COMMON,
    "lloyd_kernel": ["lloyd.cu", "round.cuh"] + _COMMON,
    "tcs_objective_kernel": ["tc_split.cu", "tc.cuh"] + _COMMON,
    "tc_objective_kernel": ["tc_objective.cu", "tc_rows.cuh", "tc.cuh"] + _COMMON,
    "tw_objective_kernel": ["tc_wide.cu", "tc_rows.cuh", "tc.cuh"] + _COMMON,
    "tcb_objective_kernel": ["tc_bf16.cu", "tc_rows.cuh", "tc.cuh", "round.cuh"] + _COMMON,
    "tcl_lloyd_kernel": ["tc_bf16.cu", "tc_rows.cuh", "tc.cuh", "round.cuh"] + _COMMON,
}


def kernel_source_hash(kernel: str | None = None) -> str:
    """Hash of the sources of one profiled kernel (KERNEL_SOURCES), or of
    every device source a benchmark step can launch (csrc/ without the
    host-side capi.cu and the cost model, which never runs in a step): a
    profile taken on other code of that kernel carries no traffic."""
    csrc = ROOT / "paper_2311_04517_gb300" / "csrc"
    if kernel is None:
        skip = ("capi.cu", "costmodel.cu", "costmodel.h")
        files = [p for p in sorted(csrc.glob("*")) if p.name not in skip]
    else:
        files = [csrc / f for f in KERNEL_SOURCES[kernel]]
    h = hashlib.sha256()
    for p in files:
        h.update(p.read_bytes())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str, kernel_name: str):
    """DRAM bytes per launch from the committed ncu summary of this workload
    whose title names the kernel that ran, if it was taken on the current
    kernel sources."""
    txt = None
    for f in sorted((ROOT / "profiles").glob(f"{kernel}_{workload}*.md")):
        t = f.read_text()
        m0 = re.match(r"#\s+(\w+)", t)
        if m0 and m0.group(1) == kernel_name:
            txt = t
            break
    if txt is None:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    hs = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", txt)
    if not m or not hs or kernel_name not in KERNEL_SOURCES or \
            hs.group(1) != kernel_source_hash(kernel_name):
        return None
    return float(m.group(1))


# ---------------------------------------------------------------------------
# clock sampling (NVML through ctypes; nvidia-smi is too coarse for short runs)
# ---------------------------------------------------------------------------
_REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
            0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
            0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
            0x100: "display_clock_setting"}


class ClockSampler:
    def __init__(self, index: int, period_s: float = 0.002):
        self.samples = []
        self.period = period_s
        self.ok = False
        self.max_mhz = None
        try:
            self.nv = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nv.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            if self.nv.nvmlDeviceGetHandleByIndex_v2(index, ctypes.byref(self.h)) != 0:
                return
            m = ctypes.c_uint()
            if self.nv.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(m)) == 0:
                self.max_mhz = m.value
            self.ok = True
        except OSError:
            pass

    def _read(self):
        mhz = ctypes.c_uint()
        rs = ctypes.c_ulonglong()
        self.nv.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(mhz))
        fn = getattr(self.nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.nv.nvmlDeviceGetCurrentClocksThrottleReasons
        fn(self.h, ctypes.byref(rs))
        return time.perf_counter(), mhz.value, rs.value

    def _loop(self):
        while not self._stop.is_set():
            self.samples.append(self._read())
            time.sleep(self.period)

    def start(self):
        if not self.ok:
            return
        self._stop = threading.Event()
        self._t = threading.Thread(target=self._loop, daemon=True)
        self._t.start()

    def stop(self):
        if self.ok:
            self._stop.set()
            self._t.join()

    def summary(self, t0: float, t1: float):
        if not self.ok:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvml unavailable"]}
        win = [s for s in self.samples if t0 <= s[0] <= t1]
        if not win:  # timed region shorter than the sampling period
            win = sorted(self.samples, key=lambda s: min(abs(s[0] - t0), abs(s[0] - t1)))[:3]
        reasons = set()
        for _, _, r in win:
            for bit, name in _REASONS.items():
                if r & bit and name != "gpu_idle":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(s[1] for s in win), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(reasons), "samples": len(win)}


# ---------------------------------------------------------------------------
def dist_count(iters, s, k, n, k_best):
    """Distances of one step: every Lloyd assignment pass (iters + 1 per
    worker) over its sample, plus the full-data objective of each group's
    best incumbent (k_best: list of their k)."""
    kb = sum(int(v) for v in k_best) if hasattr(k_best, "__len__") else int(k_best)
    return float(sum((int(i) + 1) * int(sw) * int(kw) for i, sw, kw in zip(iters, s, k))) + n * kb


def group_members(ws):
    return [np.flatnonzero(ws.group == g) for g in sorted(set(int(v) for v in ws.group))]


def workload_config(wl, strategy, args, world: int = 1):
    st = strategy if strategy != "hybrid" else f"hybrid (competitive for {n_comp(args)} rounds)"
    par = ("one GPU" if world == 1 else
           f"one job on {world} GPUs: workers in contiguous ranges per rank, the objective's "
           f"rows in blocks per rank (all-reduce), the cooperative share as an all-gather of "
           f"(f-hat, index) and a broadcast of the best incumbent")
    return {"workload": f"{wl.name}: {wl.notes}", "n": wl.n, "d": wl.d, "k": list(wl.k),
            "workers": wl.W, "s": list(wl.s), "strategy": st, "parallelism": par,
            "step": "one HPClust round for every worker + full-data objective of the best "
                    "incumbent of each sharing group (workers with equal k)",
            "l2": "inputs larger than L2 (X is %.0f MB)" % (wl.n * wl.d * 4 / 1e6),
            "lloyd_max_iter": 300, "lloyd_rel_tol": 1e-4, "kmeanspp_candidates": 3}


def job_totals(ms: float, dist_total: float, device):
    """Whole-job figures over the ranks of an initialised process group: the
    slowest rank's time and the sum of the distances every rank evaluated
    (no collective on the data path; this is the only exchange)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, dist_total
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dd = torch.tensor([dist_total], dtype=torch.float64, device=device)
    dist.all_reduce(dd)
    return float(t.item()), float(dd.item())


def bench_workload(args):
    wl = synth.workload(args.workload)
    if args.rows is not None:
        wl = replace(wl, n=int(args.rows))
    if args.workers is not None:
        wl = replace(wl, W=int(args.workers))
    return wl


def n_comp(args):
    """Hybrid strategy: the first half of the rounds competitive (the
    paper's T1 = T2); with the step count left to the bench, ten rounds past
    the warm-up."""
    if args.n_competitive is not None:
        return args.n_competitive
    if args.steps is None:
        return args.warmup + 10
    return (args.warmup + args.steps) // 2


def load_data(wl, device, seed):
    # up to 2e8 floats on the CPU (same data in both arms); larger on the GPU
    if wl.n * wl.d <= 200_000_000:
        X = synth.make_data(wl, "cpu", seed)
        return X.to(device) if device != "cpu" else X
    return synth.make_data(wl, device, seed)


def host_prefix(wl, seed, rows):
    """The first `rows` rows of the workload's data on the host, the same
    rows the GPU arm uses: drawn on the CPU up to 2e8 floats, else with the
    device generator the GPU arm uses (whole 4e6-row chunks, so the rows are
    the full data's first rows), or on the CPU (other draws of the same
    mixture) when no GPU is present."""
    if wl.n * wl.d <= 200_000_000:
        return synth.make_data(wl, "cpu", seed)[:rows].numpy(), "same rows as the GPU arm"
    chunk = 4_000_000
    n_gen = min(wl.n, -(-rows // chunk) * chunk)
    if torch.cuda.is_available():
        X = synth.make_data(wl, "cuda", seed, n=n_gen)
        out = X[:rows].cpu().numpy()
        del X
        torch.cuda.empty_cache()
        return out, "same rows as the GPU arm"
    return synth.make_data(wl, "cpu", seed, n=n_gen)[:rows].numpy(), \
        "other draws of the same mixture (no GPU for the device generator)"


class BoundedOracle:
    """A bounded sample of one step of a workload whose whole oracle step
    would take minutes (each step of the large workload evaluates about
    5e11 distances): per-component timing on the host cores.  Set-up
    (untimed): eight seed-selected workers' samples, drawn by the oracle
    from a row prefix of X, and K-means++ on the smallest of them (its time
    is reported apart).  Step r: one Lloyd update (two assignment passes and
    one update, Algorithm 1) on worker sel[r mod 8]'s sample from those
    centroids, and the full-data objective (Eq. 1) over the next block of
    `block` prefix rows."""

    def __init__(self, orc, Xp, wl, ws, seed, block=100_000):
        self.orc, self.Xp, self.block = orc, Xp, block
        rng = np.random.default_rng(seed + 4321)
        self.sel = sorted(int(w) for w in rng.choice(wl.W, min(8, wl.W), replace=False))
        self.S = {w: orc.draw_sample(Xp, seed, w, 0, int(ws.s[w]))[0] for w in self.sel}
        self.ws = ws
        w0 = min(self.sel, key=lambda w: int(ws.s[w]))
        k0 = int(ws.k[w0])
        t0 = time.perf_counter()
        kp = orc.kmeanspp(self.S[w0], np.zeros((k0, wl.d), np.float32), np.ones(k0, np.uint8),
                          3, seed, w0, 0)
        self.kpp_s = time.perf_counter() - t0
        self.kpp_worker = (w0, int(ws.s[w0]), k0)
        self.C, self.deg = kp["C"], kp["degenerate"]
        self.row = 0

    def step(self, r):
        w = self.sel[r % len(self.sel)]
        S = self.S[w]
        k = self.C.shape[0]
        self.orc.lloyd(S, self.C, self.deg, max_iter=1, rel_tol=0.0)
        a = self.row
        b = min(self.Xp.shape[0], a + self.block)
        self.orc.objective(self.Xp[a:b], self.C, self.deg)
        self.row = b if b < self.Xp.shape[0] else 0
        return 2.0 * S.shape[0] * k + float(b - a) * k

    def describe(self, steps, el):
        w0, s0, k0 = self.kpp_worker
        return (f"bounded sample: {steps} steps of one Lloyd update (2 assignment passes) on one "
                f"of 8 seed-selected workers' samples (workers {self.sel}, s = "
                f"{[int(self.ws.s[w]) for w in self.sel]}, drawn from a {self.Xp.shape[0]}-row "
                f"prefix of X) + the objective over {self.block} rows, {el:.1f} s; K-means++ "
                f"for worker {w0} (s = {s0}, k = {k0}) took {self.kpp_s:.1f} s apart")


def oracle_step_work(wl, ws):
    groups = group_members(ws)
    return (sum((10 + 1) * int(s) * int(k) for s, k in zip(ws.s, ws.k)) +
            wl.n * sum(int(ws.k[g[0]]) for g in groups)) * wl.d


def cpu_oracle_rate(X_np, wl, ws, strategy, seed, budget_s=12.0, max_rounds=5):
    """Oracle distances/s on the host cores.  Small workloads: whole steps
    (round + objectives) from the all-degenerate start.  Workloads whose one
    oracle step would take minutes: steps of BoundedOracle until the
    budget."""
    import oracle as orc
    orc.build()
    strat = {"cooperative": orc.COOPERATIVE, "hybrid": orc.HYBRID}.get(strategy, orc.COMPETITIVE)
    groups = group_members(ws)
    if oracle_step_work(wl, ws) < 2e10:
        st = orc.RoundState(wl.d, ws.s, ws.k, ws.group)
        dist = 0.0
        t0 = time.perf_counter()
        rounds = 0
        while rounds < max_rounds:
            res = orc.round_(X_np, st, strat, seed, rounds, n_competitive=max_rounds // 2)
            kb = []
            for g in groups:
                b = int(g[np.argmin(st.fhat[g])])
                C, deg = st.centroids(b)
                orc.objective(X_np, C, deg)
                kb.append(int(ws.k[b]))
            dist += dist_count(res["iters"], ws.s, ws.k, X_np.shape[0], kb)
            rounds += 1
            if time.perf_counter() - t0 > budget_s:
                break
        el = time.perf_counter() - t0
        return dist / el, el, (f"{rounds} oracle rounds from all-degenerate start "
                               f"(each: round + full-data objectives), {el:.1f} s"), orc.num_threads()
    bo = BoundedOracle(orc, X_np, wl, ws, seed)
    dist = 0.0
    steps = 0
    t0 = time.perf_counter()
    while steps < 1 or time.perf_counter() - t0 < budget_s:
        dist += bo.step(steps)
        steps += 1
    el = time.perf_counter() - t0
    return dist / el, el, bo.describe(steps, el), orc.num_threads()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as orc
    orc.build()
    K = args.steps if args.steps is not None else 5
    wl = bench_workload(args)
    ws = synth.worker_setup(wl)
    strat = {"cooperative": orc.COOPERATIVE, "hybrid": orc.HYBRID}.get(args.strategy,
                                                                       orc.COMPETITIVE)
    groups = group_members(ws)
    if oracle_step_work(wl, ws) < 2e10:
        X = load_data(wl, "cpu", wl.seed).numpy()
        st = orc.RoundState(wl.d, ws.s, ws.k, ws.group)

        def step(r):
            res = orc.round_(X, st, strat, wl.seed, r, n_competitive=n_comp(args))
            kb = []
            for g in groups:
                b = int(g[np.argmin(st.fhat[g])])
                C, deg = st.centroids(b)
                orc.objective(X, C, deg)
                kb.append(int(ws.k[b]))
            return dist_count(res["iters"], ws.s, ws.k, wl.n, kb)
        sample = f"{K} full oracle steps (round + full-data objective)"
        bo = None
    else:
        n_host = min(wl.n, max(1, 200_000_000 // wl.d))
        Xp, how = host_prefix(wl, wl.seed, n_host)
        bo = BoundedOracle(orc, Xp, wl, ws, wl.seed)
        step = bo.step

    for r in range(args.warmup):
        step(r)
    dist = 0.0
    t0 = time.perf_counter()
    for r in range(args.warmup, args.warmup + K):
        dist += step(r)
    el = time.perf_counter() - t0
    v = dist / el
    if bo is not None:
        sample = bo.describe(K, el) + f"; prefix rows: {how}"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": K, "warmup": args.warmup,
            "ms_per_step": el * 1e3 / max(1, K), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wl, args.strategy, args),
            "cpu_baseline": {"kind": "oracle", "cores": orc.num_threads(),
                             "sample": sample, "value": v, "unit": UNIT},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# Error windows of the tensor-core products, as the searches bound them: a
# computed search value lies within E = c (||x|| + max||c||)^2 of the exact
# one, and a row is proven only when its top-2 margin exceeds 2E; rows under
# it take the exact stages.  c for the built forms: TF32 2^-10, split TF32
# 2^-16, split BF16 2^-14; for one BF16 or one FP8 e4m3 product the same rule
# with their unit roundoffs (2^-8, 2^-4) gives 2^-7 and 2^-3.
WINDOW_REL = {"fp8_e4m3": 2.0 ** -3, "bf16": 2.0 ** -7, "tf32": 2.0 ** -10,
              "split_bf16": 2.0 ** -14, "split_tf32": 2.0 ** -16}


def precision_windows(X, C, deg, rows: int = 200_000, seed: int = 1):
    """Fraction of sampled rows whose exact (FP64) top-2 margin to the live
    centroids C lies inside each product's error window 2E: the rows each
    precision would have to settle exactly."""
    g = torch.Generator(device=X.device).manual_seed(seed)
    idx = torch.randint(0, X.shape[0], (min(rows, X.shape[0]),), generator=g, device=X.device)
    live = (deg == 0) if deg is not None else torch.ones(C.shape[0], dtype=torch.bool,
                                                         device=C.device)
    Cl = C[live].double()
    if Cl.shape[0] < 2:
        return None
    cmax = float(Cl.norm(dim=1).max())
    near = {k: 0 for k in WINDOW_REL}
    n = 0
    for a in range(0, idx.numel(), 20_000):
        Xs = X[idx[a:a + 20_000]].double()
        dd = torch.cdist(Xs, Cl) ** 2
        t2 = torch.topk(dd, 2, dim=1, largest=False).values
        margin = t2[:, 1] - t2[:, 0]
        R = (Xs.norm(dim=1) + cmax) ** 2
        for k, c in WINDOW_REL.items():
            near[k] += int((margin <= 2.0 * c * R).sum())
        n += Xs.shape[0]
    return {k: v / n for k, v in near.items()} | {"rows": n}


def time_to_objective(H, ctx, X, wl, ws, strategy, seed, groups, R, args, dev):
    """Wall time (CUDA events) for R rounds plus the full-data objective of
    each group's best incumbent after every round, on fresh batches: the
    plain FP32 path (CUDA-core search everywhere, rounds issued one by one)
    against the path the bench times (tensor-core search where it was
    measured faster, rounds replayed from a CUDA graph).  Reports the time at
    which each reached the plain path's final objectives (per group, within
    1e-6 relative)."""
    out = {}
    logs = {}
    samples = {}
    mode0 = args.tensor_cores
    for arm in ("fp32", "default"):
        ctx.set_tensor_cores(0 if arm == "fp32" else mode0)
        b = H.Batch(wl.d, ws.s, ws.k, ws.group, device=dev, n_competitive=n_comp(args))
        fh = torch.empty(wl.W, dtype=torch.float64).pin_memory()
        f_log = torch.zeros((R, len(groups)), dtype=torch.float64, device=dev)
        graph = None
        if arm == "default" and args.graph:
            H.hpc_round_prepare(ctx, X, b, strategy, seed, 0)
            side = torch.cuda.Stream(dev)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=side):
                ctx.set_stream(side)
                H.hpc_round_enqueue(ctx)
            ctx.set_stream(torch.cuda.current_stream(dev))
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(R + 1)]
        t0 = ctx.timestamp()                       # the device clock of t_done
        ev[0].record()
        runs = []                                  # per round: (f_new / s, t_done)
        for r in range(R):
            if graph is not None:
                graph.replay()
            else:
                H.hpc_round(ctx, X, b, strategy, seed, r)
            runs.append((b.f_new.clone(), b.t_done.clone()))
            if wl.W == 1:
                bs = [0]
            else:
                fh.copy_(b.fhat)
                bs = [int(g[np.argmin(fh.numpy()[g])]) for g in groups]
            for gi, w in enumerate(bs):
                C, deg = b.centroids(w)
                H.hpc_objective(ctx, X, C, deg, f_out=f_log[r, gi:gi + 1])
            ev[r + 1].record()
        torch.cuda.synchronize()
        ctx.check_status()
        logs[arm] = (f_log.cpu().numpy(), [ev[0].elapsed_time(e) for e in ev[1:]])
        sw = np.asarray(ws.s, np.float64)
        samples[arm] = ([f.cpu().numpy() / sw for f, _ in runs],
                        [(t.cpu().numpy() - int(t0.item())) / 1e6 for _, t in runs],
                        float(b.fhat.min().item()))
        del graph
    ctx.set_tensor_cores(mode0)
    target = logs["fp32"][0][-1]
    for arm, (f, t) in logs.items():
        hit = [r for r in range(R) if np.all(f[r] <= target * (1 + 1e-6))]
        out[f"{arm}_ms"] = t[hit[0]] if hit else None
        out[f"{arm}_rounds"] = hit[0] + 1 if hit else None
    out["speedup"] = (out["fp32_ms"] / out["default_ms"]) if out["default_ms"] else None
    out["final_objectives_rel_diff"] = float(np.max(np.abs(logs["default"][0][-1] - target)
                                                    / target))
    # Section 6.4's baseline convergence time: the baseline sample objective
    # is the worse of the two paths' best sample objectives per point (the
    # largest over the compared algorithms, one run each), and t-bar the time
    # from the first round's start until any worker's run first ends at or
    # below it (device clock, stamped where each run ends)
    fbar = max(v[2] for v in samples.values())
    for arm, (fv, tv, _) in samples.items():
        hits = [float(t[w]) for f, t in zip(fv, tv) for w in range(len(f)) if f[w] <= fbar]
        out[f"{arm}_tbar_ms"] = min(hits) if hits else None
    out["baseline_sample_objective_per_point"] = fbar
    out["tbar_speedup"] = (out["fp32_tbar_ms"] / out["default_tbar_ms"]
                           if out["fp32_tbar_ms"] and out["default_tbar_ms"] else None)
    out.update({"rounds": R, "target": "the plain FP32 path's full-data objective of each "
                "group's best incumbent after the last round, within 1e-6 relative",
                "fp32_path": "CUDA-core search, rounds issued one by one",
                "default_path": "the bench's path: objective search form per (d, k) as tuned, "
                                "rounds replayed from a CUDA graph"})
    return out


def run_mine(args):
    from paper_2311_04517_gb300 import hpclust as H
    from paper_2311_04517_gb300 import costmodel as CM
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist_ok = world > 1
    if dist_ok:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    from paper_2311_04517_gb300 import multirank as MR
    wl = bench_workload(args)
    ws = synth.worker_setup(wl)
    # one job on every rank: the same data, the workers split into
    # contiguous ranges (each with its global random streams), the full-data
    # objective split into row blocks
    seed = wl.seed
    X = load_data(wl, dev, seed)
    strategy = {"cooperative": H.HPC_COOPERATIVE, "hybrid": H.HPC_HYBRID}.get(
        args.strategy, H.HPC_COMPETITIVE)
    ctx = H.Context(local)
    ctx.set_tensor_cores(args.tensor_cores)
    ranges = MR.worker_ranges(ws.s, ws.k, world)
    w0, w1 = ranges[rank]
    if w1 <= w0:
        raise SystemExit(f"rank {rank}: more ranks than workers ({wl.W})")
    lw = slice(w0, w1)
    Wl = w1 - w0
    batch = H.Batch(wl.d, ws.s[lw], ws.k[lw], ws.group[lw], device=dev,
                    n_competitive=n_comp(args), worker0=w0)
    job = MR.RankedRun(MR.LibraryBackend(ctx, X, batch), ws.s, ws.k, ws.group, wl.d, w0, w1,
                       device=dev)
    ra, rb = MR.row_range(wl.n, world, rank) if world > 1 else (0, wl.n)
    Xo = X[ra:rb]          # this rank's rows of the full-data objective
    groups = group_members(ws)
    f_sse = torch.zeros(len(groups), dtype=torch.float64, device=dev)
    Wm = args.warmup
    best_log = []
    fhat_host = torch.empty(Wl, dtype=torch.float64).pin_memory()

    def bests():
        # the incumbent with the smallest objective per sample point in each
        # group (one worker: no read-back needed)
        if wl.W == 1:
            return [0]
        fhat_host.copy_(batch.fhat)
        fh = fhat_host.numpy()
        return [int(g[np.argmin(fh[g])]) for g in groups]

    def best_centroids():
        """(k, C, flags) of each sharing group's best incumbent: on one rank
        from the batch, across ranks by the all-gather and broadcast of the
        cooperative share (which synchronises with the round)."""
        if world == 1:
            return [(int(ws.k[b]),) + tuple(batch.centroids(b)) for b in bests()]
        out = []
        for key in range(len(job.keys)):
            _, _, C, deg = job.best(ranges, key)
            kb = job.keys[key][1]
            out.append((kb, C.view(kb, wl.d), deg))
        return out

    graph = None
    graph_launches = 0
    # CUDA events around every launch of a round (graph nodes when recorded
    # in the graph): per-phase device times of each step
    ctx.set_phase_timing(True)
    if args.graph and not (world > 1 and strategy != H.HPC_COMPETITIVE):
        # one round recorded once; its round index lives on the device and
        # advances with every replay (rounds 0, 1, 2, ... as below)
        H.hpc_round_prepare(ctx, X, batch, strategy, seed, 0)
        side = torch.cuda.Stream(dev)
        graph = torch.cuda.CUDAGraph()
        l0 = ctx.launch_count()
        with torch.cuda.graph(graph, stream=side):
            ctx.set_stream(side)
            H.hpc_round_enqueue(ctx)
        ctx.set_stream(torch.cuda.current_stream(dev))
        graph_launches = ctx.launch_count() - l0

    # across ranks the cooperative share is an exchange between rounds
    shared = world > 1 and strategy != H.HPC_COMPETITIVE

    def run_round(r):
        if shared:
            job.round(strategy, seed, r, ranges, n_competitive=n_comp(args))
        elif graph is not None:
            graph.replay()
        else:
            H.hpc_round(ctx, X, batch, strategy, seed, r)

    phase_log = []

    def step(r, log_row=None, ev=None):
        run_round(r)
        if log_row is not None:
            iters_log[log_row].copy_(batch.iters, non_blocking=True)
        cb = best_centroids()
        if log_row is not None:
            best_log.append([kb for kb, _, _ in cb])
            if wl.W > 1:
                # best_centroids() has synchronised with the round: its phase
                # times are ready (read before the next replay re-records them)
                phase_log.append(ctx.phase_times())
        if ev is not None:
            ev[0].record()
        for gi, (kb, C, deg) in enumerate(cb):
            H.hpc_objective(ctx, Xo, C, deg, f_out=f_sse[gi:gi + 1])
        if world > 1:
            dist.all_reduce(f_sse)     # Eq. 1 is a sum over the ranks' rows
        if ev is not None:
            ev[1].record()

    t_warm = 0.0
    for r in range(Wm):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        step(r)
        torch.cuda.synchronize(dev)
        t_warm = time.perf_counter() - t0
    ctx.check_status()
    if args.steps is not None:
        K = args.steps
    else:
        # about TIMED_BUDGET_S of timed steps (the slowest rank's estimate)
        tw = torch.tensor([t_warm], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(tw, op=dist.ReduceOp.MAX)
        K = int(min(100, max(5, TIMED_BUDGET_S / max(float(tw.item()), 1e-6))))
    iters_log = torch.zeros((K, Wl), dtype=torch.int32, device=dev)
    # the objective's search form per (d, k), measured on this data with the
    # incumbents the warm-up rounds produced (outside the timed steps)
    forms = {}
    if args.autotune and args.tensor_cores == 2:
        rows = min(wl.n, max(1, 512_000_000 // (4 * wl.d)))   # a prefix larger than L2
        # beside it, the search guided by the shipped cost model (what it
        # would pick and how many forms it times); the exhaustive choice stays
        cm_params = None
        if CM.OUT.exists():
            cm_params = torch.tensor(json.loads(CM.OUT.read_text())["params"],
                                     dtype=torch.float32, device=dev)
        for kb, C, deg in best_centroids():
            if kb in forms:
                continue
            form, tms = ctx.autotune_objective(X[:rows], C, deg, reps=3)
            forms[kb] = {"form": H.SEARCH_NAMES[form], "ms_per_call": tms, "rows": rows}
            if cm_params is not None:
                gform, gms, timed = ctx.autotune_objective_guided(X[:rows], C, cm_params, deg,
                                                                  reps=3, margin=CM.MARGIN)
                ctx.set_objective_form(wl.d, kb, form)
                forms[kb]["guided"] = {"form": H.SEARCH_NAMES[gform], "forms_timed": timed,
                                       "forms_built": len(tms), "ms_per_call": gms}
    torch.cuda.synchronize()
    if dist_ok:
        dist.barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(K)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.01)
    launches0 = ctx.launch_count()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    start.record()
    for i in range(K):
        step(Wm + i, i, evs[i])
    end.record()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    clocks.stop()
    launches = ctx.launch_count() - launches0 + graph_launches * K
    st = ctx.sync_status()
    if st != 0:
        raise RuntimeError(f"device status {st}")
    if not phase_log:
        # one worker: no per-step synchronisation inside the timed region, so
        # the phase times come from a few more steps after it
        extra_iters = []
        for i in range(min(K, 10)):
            run_round(Wm + K + i)
            phase_log.append(ctx.phase_times())
            extra_iters.append(batch.iters.cpu().numpy().copy())
        Wm_extra = min(K, 10)
    else:
        Wm_extra = 0
    ms = start.elapsed_time(end)
    obj_ms = [a.elapsed_time(b) for a, b in evs]
    iters = iters_log.cpu().numpy()
    dist_total = sum(dist_count(iters[i], ws.s[lw], ws.k[lw], rb - ra, best_log[i])
                     for i in range(K))
    ms, dist_total = job_totals(ms, dist_total, dev)
    value = dist_total / (ms / 1e3)

    # end to end: host-resident (pinned) data copied in every step, results
    # read back; about 30 s of steps at most (a step copies all of X)
    copy_s = wl.n * wl.d * 4 / 200e9
    E = args.e2e_steps if args.e2e_steps is not None else max(
        3, min(K, 20, int(30.0 / (ms / K / 1e3 + copy_s))))
    e2e = None
    if E > 0:
        X_host = torch.empty(X.shape, dtype=X.dtype, pin_memory=True)
        X_host.copy_(X)
        res_host = torch.empty(len(groups) * 8 + Wl, dtype=torch.float64).pin_memory()
        C_host = torch.empty_like(batch.C, device="cpu").pin_memory()
        e_iters = torch.zeros((E, Wl), dtype=torch.int32, device=dev)
        e_best = []
        r0 = Wm + K + Wm_extra
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # Each step copies its X in row chunks; the objective of the current
        # best incumbents runs on every chunk as soon as it has arrived (it is
        # a sum over rows); the round then runs on the complete X.  With room
        # for a second copy of X on the device, the copies alternate between
        # two buffers and step i + 1's copy runs during step i's work (its
        # buffer is free once step i - 1's round is done); otherwise a step's
        # copy waits for the previous step.  Work per step: one full copy,
        # one full objective per group, one round.
        nck = 8
        rows = (wl.n + nck - 1) // nck
        rows = (rows + 3) // 4 * 4                      # 16-byte aligned chunk starts
        bufs = [X]
        free_b, _ = torch.cuda.mem_get_info(dev)
        if free_b > X.numel() * 4 + (8 << 30):
            bufs.append(torch.empty_like(X))
        nb = len(bufs)
        f_chunks = torch.zeros((len(groups), nck), dtype=torch.float64, device=dev)
        main = torch.cuda.current_stream(dev)
        copy_stream = torch.cuda.Stream(dev)
        arrived = [[torch.cuda.Event() for _ in range(nck)] for _ in range(nb)]
        freed = [torch.cuda.Event() for _ in range(nb)]

        # per-step and per-copy device times and the clocks of the e2e steps
        diag = {"copy": [], "step": []}

        def timing_event(stream):
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
            return ev

        def issue_copy(i):
            bi = i % nb
            if nb == 1:
                copy_stream.wait_stream(main)           # X is free once the last step is done
            else:
                copy_stream.wait_event(freed[bi])       # the last round on this buffer is done
            c0 = timing_event(copy_stream)
            with torch.cuda.stream(copy_stream):
                for c in range(nck):
                    a, b_ = c * rows, min(wl.n, (c + 1) * rows)
                    if a < b_:
                        bufs[bi][a:b_].copy_(X_host[a:b_], non_blocking=True)
                    arrived[bi][c].record(copy_stream)
            diag["copy"].append((c0, timing_event(copy_stream)))

        def round_on(buf, r):
            if nb == 1:
                run_round(r)
            elif shared:
                job.b.X = buf
                job.round(strategy, seed, r, ranges, n_competitive=n_comp(args))
            else:
                H.hpc_round(ctx, buf, batch, strategy, seed, r)

        def e2e_steps(n_steps, r_first, timed):
            issue_copy(0)
            for i in range(n_steps):
                if nb == 2 and i + 1 < n_steps:
                    issue_copy(i + 1)
                e2e_step(i, r_first + i, timed)
                if nb == 1 and i + 1 < n_steps:
                    issue_copy(i + 1)

        def e2e_step(i, r, timed):
            bi = i % nb
            cb = best_centroids()
            if timed:
                e_best.append([kb for kb, _, _ in cb])
                diag["step"].append(timing_event(main))
            f_chunks.zero_()
            for c in range(nck):
                # the chunk's rows within this rank's block of the objective
                a, b_ = max(ra, c * rows), min(rb, (c + 1) * rows)
                main.wait_event(arrived[bi][c])
                if a >= b_:
                    continue
                for gi, (kb, C, deg) in enumerate(cb):
                    H.hpc_objective(ctx, bufs[bi][a:b_], C, deg, f_out=f_chunks[gi, c:c + 1])
            round_on(bufs[bi], r)
            freed[bi].record(main)
            if timed:
                e_iters[i].copy_(batch.iters, non_blocking=True)
            # per-chunk objectives are read back and added on the host
            res_host[:len(groups) * nck].copy_(f_chunks.view(-1), non_blocking=True)
            res_host[len(groups) * nck:].copy_(batch.fhat, non_blocking=True)
            C_host.copy_(batch.C, non_blocking=True)

        # one untimed step first: the call path's first use on this context
        # sets up its scratch and pinned staging (the timed steps above ran
        # the recorded graph)
        e2e_steps(1, r0, False)
        torch.cuda.synchronize()
        eclk = ClockSampler(local)
        eclk.start()
        te0 = time.perf_counter()
        e0.record()
        e2e_steps(E, r0 + 1, True)
        e1.record()
        torch.cuda.synchronize()
        te1 = time.perf_counter()
        eclk.stop()
        e_ms = e0.elapsed_time(e1)
        try:
            marks = diag["step"] + [e1]
            step_ms = [marks[i].elapsed_time(marks[i + 1]) for i in range(E)]
            copy_ms = [a.elapsed_time(b) for a, b in diag["copy"][-E:]]
            e_diag = {"step_ms": {"min": float(min(step_ms)),
                                  "median": float(statistics.median(step_ms)),
                                  "max": float(max(step_ms))},
                      "copy_ms_median": float(statistics.median(copy_ms)),
                      "clocks": eclk.summary(te0, te1)}
        except Exception as exc:  # a diagnostic only
            e_diag = {"error": str(exc)}
        ei = e_iters.cpu().numpy()
        e_dist = sum(dist_count(ei[i], ws.s[lw], ws.k[lw], rb - ra, e_best[i]) for i in range(E))
        e_ms, e_dist = job_totals(e_ms, e_dist, dev)
        e_value = e_dist / (e_ms / 1e3)
        if shared:
            job.b.X = X
        # its own steps (later rounds than the timed ones: fewer Lloyd updates
        # as the incumbents improve, so the copy of X weighs more)
        e2e = {"value": e_value, "unit": UNIT, "device_buffers": nb, "steps": E,
               "ms_per_step": e_ms / E, "lloyd_iters_mean": float(ei.mean()), **e_diag,
               "h2d_bytes_per_step": int(X_host.numel() * 4),
               "d2h_bytes_per_step": int(res_host.numel() * 8 + C_host.numel() * 4 +
                                         (Wl * 8 if wl.W > 1 else 0))}
        del X_host, bufs

    hbm, src = peaks()
    obj_avg_ms = float(np.mean(obj_ms)) / len(groups)  # one launch per group per step
    kb0 = int(best_log[0][0]) if best_log else int(ws.k[0])
    k_mean = float(np.mean(best_log[0])) if best_log else float(kb0)
    form0 = ctx.objective_form(wl.n, wl.d, kb0)
    obj_kernel = {H.HPC_SEARCH_SIMT: "objective_kernel",
                  H.HPC_SEARCH_SPLIT_TF32: "tcs_objective_kernel",
                  H.HPC_SEARCH_TF32: "tc_objective_kernel" if kb0 <= 128
                  else "tw_objective_kernel",
                  H.HPC_SEARCH_SPLIT_BF16: "tcb_objective_kernel"}[form0]
    obj_entry = roofline_entry(obj_kernel, H.SEARCH_NAMES[form0], rb - ra, wl.d, k_mean,
                               obj_avg_ms, hbm, src,
                               profiled_traffic("objective", wl.name, obj_kernel))
    # the Lloyd launches of the timed steps (their phase times: one launch
    # per 128 workers per step)
    chunks = (wl.W + 127) // 128
    lloyd_ms = [p["lloyd"] for p in phase_log]
    lsched = ctx.lloyd_schedule(int(max(ws.s)), wl.d, int(max(ws.k)))
    lloyd_kernel_name = "lloyd_kernel" if lsched["form"] == "simt" else "tcl_lloyd_kernel"
    if Wm_extra:
        it_rows = [(int(it[w]) + 1, int(ws.s[w0 + w]), int(ws.k[w0 + w]))
                   for it in extra_iters for w in range(Wl)]
    else:
        it_rows = [(int(iters[i][w]) + 1, int(ws.s[w0 + w]), int(ws.k[w0 + w]))
                   for i in range(K) for w in range(Wl)]
    lloyd_entry = lloyd_roofline(lloyd_kernel_name, lsched["form"], it_rows, wl.d,
                                 len(lloyd_ms) * chunks,
                                 float(np.sum(lloyd_ms)) / (len(lloyd_ms) * chunks), hbm, src,
                                 profiled_traffic("lloyd", wl.name, lloyd_kernel_name))
    # how far the last step's CTA plan was from an even spread of the work
    lplan = None
    if lsched["form"] == "split_bf16" and 1 < Wl <= 128 and K >= 2 and not Wm_extra:
        try:
            lplan = plan_balance(ws.s[w0:w0 + Wl], ws.k[w0:w0 + Wl], iters[K - 2], iters[K - 1],
                                 int(lsched["blocks"]))
        except Exception as exc:  # a diagnostic only
            lplan = {"error": str(exc)}
    phase_ms = {k: float(np.mean([p[k] for p in phase_log])) for k in phase_log[0]}
    phase_ms["objective"] = float(np.mean(obj_ms))
    # the roofline line names the kernel that takes the larger share of a step
    lloyd_step_ms = phase_ms["lloyd"]
    dominant, other = ((lloyd_entry, obj_entry) if lloyd_step_ms > phase_ms["objective"]
                       else (obj_entry, lloyd_entry))
    tto = None
    R = args.tto_rounds if args.tto_rounds is not None else min(wl.rounds, 10)
    if R > 0 and world == 1:
        tto = time_to_objective(H, ctx, X, wl, ws, strategy, seed, groups, R, args, dev)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": Wm, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(wl, args.strategy, args, world),
            "round_issue": ("one round recorded in a CUDA graph, replayed every step" if args.graph
                            else "calls issued one by one"),
            "roofline": dominant,
            "roofline_other": other,
            "phase_ms_per_step": phase_ms,
            "lloyd_schedule": lsched,
            "lloyd_plan_last_step": lplan,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks.summary(t0, t1),
            "lloyd_iters_mean": float(iters.mean())}
    if forms:
        line["objective_forms"] = {str(k): v for k, v in forms.items()}
    if world == 1:
        # the rows each product precision would leave to the exact stages,
        # on the first group's best incumbent after the timed steps
        kb, Cb, db = best_centroids()[0]
        line["precision_windows"] = precision_windows(X, Cb, db)
    # the stages of the tensor-core searches over one more step (rounds
    # issued directly: a recorded round keeps the counting it was recorded
    # with)
    ctx.set_search_stats(True)
    ctx.search_stats(reset=True)
    if shared:
        run_round(Wm + K + Wm_extra + (E + 1 if E > 0 else 0))
    else:
        H.hpc_round(ctx, X, batch, strategy, seed, Wm + K + Wm_extra + (E + 1 if E > 0 else 0))
    for kb, Cb, db in best_centroids():
        H.hpc_objective(ctx, Xo, Cb, db)
    line["search_stats_one_step"] = ctx.search_stats(reset=True)
    ctx.set_search_stats(False)
    if tto is not None:
        line["time_to_objective"] = tto
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the host copy for the oracle: whole X up to 2e8 floats, else a row prefix
        n_host = wl.n if wl.n * wl.d <= 200_000_000 else max(1, 200_000_000 // wl.d)
        rate, el, sample, cores = cpu_oracle_rate(X[:n_host].cpu().numpy(), wl, ws, args.strategy,
                                                  seed)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist_ok:
        dist.destroy_process_group()


def run_scaling_experiment(args):
    """Section 6.8 on one GPU: for m = 3^(i+7) points (10 blobs in 10 dims
    plus 500 noise points), eight workers with k = 10 and s = min(5000,
    m - 1000), each strategy for R rounds issued one by one (hybrid:
    competitive for the first R/2, the paper's T1 = T2 = T/2).  Reports, per
    strategy: t, the device time from the first round's start to the end of
    the run that last replaced the final best worker's incumbent (the
    paper's clustering time: the last solution update of the best worker);
    the device time of all R rounds; and eps = 100 (f - f0) / f0 of the
    full-data objective of the best incumbent against f0, the objective of
    the ten generating means (the paper states eps against the best known
    objective; the generating means stand in for it here)."""
    from paper_2311_04517_gb300 import hpclust as H
    torch.cuda.set_device(0)
    ctx = H.Context(0)
    R = args.scaling_rounds
    names = {H.HPC_COMPETITIVE: "competitive", H.HPC_COOPERATIVE: "cooperative",
             H.HPC_HYBRID: "hybrid"}
    rows = []
    for i in range(9):
        wl = synth.scaling_workload(i)
        ws = synth.worker_setup(wl)
        X = synth.scaling_data(i, "cuda", wl.seed)
        mu, _ = synth.scaling_params(wl.seed)
        f0 = float(H.hpc_objective(ctx, X, mu.float().cuda()).item())
        row = {"i": i, "m": 3 ** (i + 7), "n": wl.n, "s": int(ws.s[0]), "f_means": f0}
        for strat, name in names.items():
            batch = H.Batch(wl.d, ws.s, ws.k, ws.group, n_competitive=R // 2)
            torch.cuda.synchronize()
            t0 = ctx.timestamp()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            log = []
            for r in range(R):
                H.hpc_round(ctx, X, batch, strat, wl.seed, r)
                log.append((batch.accepted.clone(), batch.t_done.clone()))
            e1.record()
            torch.cuda.synchronize()
            ctx.check_status()
            best = int(torch.argmin(batch.fhat).item())
            C, deg = batch.centroids(best)
            f = float(H.hpc_objective(ctx, X, C, deg).item())
            acc = [r for r in range(R) if bool(log[r][0][best].item())]
            last = acc[-1] if acc else 0
            t_ms = (int(log[last][1][best].item()) - int(t0.item())) / 1e6
            row[name] = {"t_ms": t_ms, "rounds_ms": e0.elapsed_time(e1),
                         "eps_pct": 100.0 * (f - f0) / f0, "last_update_round": last}
        rows.append(row)
        del X
        torch.cuda.empty_cache()
    print(json.dumps({"experiment": "Section 6.8 scaling", "rounds": R, "workers": 8,
                      "rows": rows}), flush=True)
    ctx.close()


def main():
    args = parse_args()
    if args.scaling_experiment:
        run_scaling_experiment(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_mine(args)


if __name__ == "__main__":
    main()
