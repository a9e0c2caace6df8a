"""Seeded synthetic inputs: Gaussian-mixture data sets and worker set-ups.

This module only generates inputs; it holds none of the clustering method's
arithmetic, and both the GPU path and the CPU oracle may consume what it
makes.  The paper evaluates on 19 public data sets that are not available
here; these mixtures stand in for them, with the shapes of the workloads the
library is measured on (n rows, d dims, number of components, spread and
weights as listed in WORKLOADS), plus the paper's own synthetic scaling set
(Section 6.8: 10 blobs in (-40, 40)^10 with sd in (0, 10), 3^(i+7) points,
500 uniform noise points in (-50, 50)^10).

Mixture parameters come from a CPU torch generator seeded with ``seed``;
points are drawn chunk by chunk (component index, then mean + sd * N(0, I))
on the requested device with a generator seeded from ``seed`` as well, so a
given (workload, seed, device) always gives the same data.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch


@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    d: int
    comps: int
    means: tuple          # ("uniform", lo, hi) or ("normal", sd)
    sd: tuple             # ("const", v) or ("uniform", lo, hi)
    weights: str          # "equal", "dirichlet1", "zipf1.1"
    k: tuple              # cluster counts cycled over workers
    W: int                # workers
    s: tuple              # ("const", s) or ("uniform", lo, hi)
    rounds: int
    seed: int = 0
    notes: str = ""


WORKLOADS = {
    "tiny": Workload("tiny", 20_000, 2, 5, ("uniform", -10.0, 10.0), ("const", 1.0), "equal",
                     (5,), 1, ("const", 2_000), 20, 0,
                     "plain method, tiny: 5 isotropic Gaussians in the plane"),
    "fp32": Workload("fp32", 10_000_000, 16, 25, ("uniform", -10.0, 10.0), ("uniform", 0.5, 2.0),
                     "dirichlet1", (25,), 1, ("const", 100_000), 30, 0,
                     "plain FP32 path: 25 Gaussians in 16 dims, Dirichlet(1) weights"),
    "precision": Workload("precision", 20_000_000, 128, 100, ("normal", 5.0), ("const", 1.0),
                          "equal", (100,), 1, ("const", 250_000), 10, 0,
                          "precision: 100 Gaussians in 128 dims"),
    "batching": Workload("batching", 50_000_000, 32, 50, ("uniform", -20.0, 20.0),
                         ("uniform", 0.5, 3.0), "equal", (10, 25, 50, 100), 64,
                         ("uniform", 16_384, 262_144), 10, 0,
                         "batching: 64 workers with uneven s and k"),
    "large": Workload("large", 200_000_000, 64, 500, ("normal", 4.0), ("uniform", 0.5, 2.0),
                      "zipf1.1", (500,), 128, ("uniform", 65_536, 1_048_576), 5, 0,
                      "large: 500 Gaussians in 64 dims, Zipf(1.1) weights, 51 GB"),
}


def workload(name: str) -> Workload:
    """A named workload: one of WORKLOADS, or "scaling<i>" (Section 6.8, i = 0..8)."""
    if name.startswith("scaling"):
        return scaling_workload(int(name[len("scaling"):] or 8))
    return WORKLOADS[name]


def mixture_params(wl: Workload, seed: int | None = None):
    """Means (comps x d), sds (comps) and weights (comps), float64 on the CPU."""
    g = torch.Generator().manual_seed(wl.seed if seed is None else seed)
    m, d = wl.comps, wl.d
    if wl.means[0] == "uniform":
        lo, hi = wl.means[1], wl.means[2]
        mu = lo + (hi - lo) * torch.rand(m, d, generator=g, dtype=torch.float64)
    else:
        mu = wl.means[1] * torch.randn(m, d, generator=g, dtype=torch.float64)
    if wl.sd[0] == "const":
        sd = torch.full((m,), wl.sd[1], dtype=torch.float64)
    else:
        sd = wl.sd[1] + (wl.sd[2] - wl.sd[1]) * torch.rand(m, generator=g, dtype=torch.float64)
    if wl.weights == "equal":
        w = torch.full((m,), 1.0 / m, dtype=torch.float64)
    elif wl.weights == "dirichlet1":
        e = -torch.log(torch.rand(m, generator=g, dtype=torch.float64).clamp_min(1e-300))
        w = e / e.sum()
    elif wl.weights == "zipf1.1":
        r = torch.arange(1, m + 1, dtype=torch.float64)
        w = r ** -1.1
        w = w / w.sum()
    else:
        raise ValueError(wl.weights)
    return mu, sd, w


def make_data(wl: Workload | str, device="cpu", seed: int | None = None, n: int | None = None,
              chunk: int = 4_000_000, out: torch.Tensor | None = None) -> torch.Tensor:
    """n x d float32 mixture sample (n defaults to the workload's)."""
    if isinstance(wl, str):
        wl = workload(wl)
    seed = wl.seed if seed is None else seed
    if wl.means[0] == "scaling":
        return scaling_data(wl.means[1], device, seed)
    n = wl.n if n is None else n
    device = torch.device(device)
    mu, sd, w = mixture_params(wl, seed)
    mu32 = mu.to(device=device, dtype=torch.float32)
    sd32 = sd.to(device=device, dtype=torch.float32)
    cdf = torch.cumsum(w, 0)
    cdf = (cdf / cdf[-1]).to(device=device, dtype=torch.float64)
    g = torch.Generator(device=device).manual_seed(int(seed) * 7919 + 1)
    X = out if out is not None else torch.empty((n, wl.d), dtype=torch.float32, device=device)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        u = torch.rand(b - a, generator=g, device=device, dtype=torch.float64)
        comp = torch.searchsorted(cdf, u, right=True).clamp_max(wl.comps - 1)
        z = torch.randn((b - a, wl.d), generator=g, device=device, dtype=torch.float32)
        X[a:b] = mu32[comp] + sd32[comp, None] * z
    return X


def scaling_params(seed: int = 0):
    """The Section 6.8 blobs: means (10 x 10, uniform in (-40, 40)) and sds
    (10, uniform in (0, 10)), float64 on the CPU."""
    g = torch.Generator().manual_seed(seed)
    mu = -40 + 80 * torch.rand(10, 10, generator=g, dtype=torch.float64)
    sd = 10 * torch.rand(10, generator=g, dtype=torch.float64)
    return mu, sd


def scaling_data(i: int, device="cpu", seed: int = 0) -> torch.Tensor:
    """Section 6.8 scaling set: 10 blobs in (-40, 40)^10, sd ~ U(0, 10),
    m = 3^(i+7) points, plus 500 uniform noise points in (-50, 50)^10
    (the noise rows last)."""
    m = 3 ** (i + 7)
    device = torch.device(device)
    mu, sd = scaling_params(seed)
    mu, sd = mu.to(device), sd.to(device)
    gd = torch.Generator(device=device).manual_seed(int(seed) * 7919 + 3)
    X = torch.empty((m + 500, 10), dtype=torch.float32, device=device)
    chunk = 4_000_000
    for a in range(0, m, chunk):
        b = min(m, a + chunk)
        comp = torch.randint(0, 10, (b - a,), generator=gd, device=device)
        z = torch.randn((b - a, 10), generator=gd, device=device, dtype=torch.float64)
        X[a:b] = (mu[comp] + sd[comp, None] * z).float()
    X[m:] = (-50 + 100 * torch.rand((500, 10), generator=gd, device=device,
                                    dtype=torch.float64)).float()
    return X


def scaling_workload(i: int) -> Workload:
    """The Section 6.8 experiment as a workload: k = 10 (the blob count),
    s = min(5000, m - 1000), eight workers (the paper's CPU count)."""
    m = 3 ** (i + 7)
    return Workload(f"scaling{i}", m + 500, 10, 10, ("scaling", i), ("uniform", 0.0, 10.0),
                    "equal", (10,), 8, ("const", min(5000, m - 1000)), 10, 0,
                    f"Section 6.8 scaling set, m = 3^{i + 7} = {m} points + 500 noise points")


@dataclass
class WorkerSetup:
    s: np.ndarray
    k: np.ndarray
    group: np.ndarray


def worker_setup(wl: Workload | str, seed: int | None = None, W: int | None = None) -> WorkerSetup:
    """Per-worker sample sizes, cluster counts and sharing groups (workers
    with the same k share one group)."""
    if isinstance(wl, str):
        wl = workload(wl)
    W = wl.W if W is None else W
    rng = np.random.default_rng((wl.seed if seed is None else seed) + 1234)
    if wl.s[0] == "const":
        s = np.full(W, wl.s[1], dtype=np.int64)
    else:
        s = rng.integers(wl.s[1], wl.s[2] + 1, size=W, dtype=np.int64)
    k = np.array([wl.k[w % len(wl.k)] for w in range(W)], dtype=np.int32)
    kinds = sorted(set(int(v) for v in k))
    group = np.array([kinds.index(int(v)) for v in k], dtype=np.int32)
    return WorkerSetup(s, k, group)
