"""One HPClust job on several ranks (one process per GPU).

The method shards along its two axes (Section 4):

* Workers.  The workers of Algorithms 3-5 are independent but for the
  cooperative share.  Rank r runs the contiguous range [w0, w1) of the global
  workers (split so that each range carries about the same sample work
  sum s_w k_w); each local batch has ``worker0 = w0`` so that worker w draws
  from the random stream of its global index, whatever the split.
  - Competitive rounds (Algorithm 3) need no exchange.
  - Cooperative rounds (Algorithm 4, synchronous reading): at the start of a
    round every rank reports, per sharing group (equal group and k), its
    best incumbent (smallest f-hat per point, lowest global index on ties);
    one all-gather of those (f-hat, index) pairs gives every rank the global
    best, and its owner broadcasts that incumbent's k x d centroids and
    flags.  Each rank then runs its workers from that base: it writes the
    base over its workers' incumbent slots, runs the round's competitive
    form (base = own slot), and puts back the previous incumbent of every
    worker whose result was not accepted (the incumbent rule compares with
    the worker's own f-hat, which the base never touches).
  - Hybrid rounds (Algorithm 5) take the competitive form for rounds below
    n_competitive and the cooperative one after.
* Rows.  The full-data objective (Eq. 1) is a sum over rows: each rank takes
  its contiguous block of rows and one all-reduce adds the FP64 partials.

The collectives are torch.distributed's (NCCL between GPUs, gloo on CPU);
with no process group, or a group of one, every exchange is local.  The
compute goes through a backend with the small interface below, so the same
driver runs the CUDA library (LibraryBackend) or, in tests, a CPU reference.

Backend interface:
  pools() -> (C_pool float32 tensor, deg_pool uint8 tensor, fhat float64 tensor)
  offsets() -> (C_off, K_off): each local worker's place in the pools
  run_round(seed, round)   one competitive round of the local workers
  accepted() -> bool numpy array of the last round's incumbent decisions
  objective(rows, C, deg) -> float64 scalar tensor (Eq. 1 over `rows`)
"""
from __future__ import annotations

import numpy as np
import torch

COMPETITIVE, COOPERATIVE, HYBRID = 0, 1, 2


def worker_ranges(s, k, world: int):
    """Contiguous worker ranges [(w0, w1)] for `world` ranks, each carrying
    about the same share of sum_w s_w k_w; every rank gets at least one
    worker while there are as many workers as ranks."""
    s = np.asarray(s, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    W = len(s)
    if world < 1:
        raise ValueError("world >= 1")
    work = np.cumsum(s * k) if W else np.zeros(0)
    total = float(work[-1]) if W else 0.0
    bounds = [0]
    for r in range(1, world):
        # end of rank r - 1's range: the first prefix that reaches r / world
        # of the total work
        b = int(np.searchsorted(work, total * r / world, side="left")) + 1 if W else 0
        if W >= world:
            b = min(max(b, bounds[-1] + 1), W - (world - r))
        else:
            b = min(max(b, bounds[-1]), W)
        bounds.append(b)
    bounds.append(W)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def row_range(n: int, world: int, rank: int):
    """Contiguous rows [a, b) of rank `rank` (16-byte aligned starts for
    rows of 4-byte values when n allows)."""
    per = -(-n // world)
    per = (per + 3) // 4 * 4
    a = min(n, rank * per)
    return a, min(n, a + per)


class RankedRun:
    """The rank's part of one job: its workers [w0, w1) of a run with global
    sample sizes s, cluster counts k and groups `group`, and dimension d."""

    def __init__(self, backend, s, k, group, d: int, w0: int, w1: int, pg=None,
                 device=None):
        self.b = backend
        self.s = np.asarray(s, dtype=np.int64)
        self.k = np.asarray(k, dtype=np.int32)
        self.group = (np.zeros(len(self.s), np.int32) if group is None
                      else np.asarray(group, dtype=np.int32))
        self.d = int(d)
        self.w0, self.w1 = int(w0), int(w1)
        self.pg = pg
        self.device = device if device is not None else torch.device("cpu")
        # pool offsets of the local workers
        if self.w1 > self.w0:
            co, ko = backend.offsets()
            self.C_off = [int(v) for v in co]
            self.K_off = [int(v) for v in ko]
        else:
            self.C_off, self.K_off = [], []
        # sharing groups of the whole run: workers with equal group and k
        keys = sorted({(int(g), int(kk)) for g, kk in zip(self.group, self.k)})
        self.keys = keys
        self.key_of = {w: keys.index((int(self.group[w]), int(self.k[w])))
                       for w in range(len(self.s))}

    # ---- collectives (local when there is no group of several ranks) ----
    def _dist(self):
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized() and \
                dist.get_world_size(self.pg) > 1:
            return dist
        return None

    def _all_gather(self, t):
        dist = self._dist()
        if dist is None:
            return [t]
        out = [torch.empty_like(t) for _ in range(dist.get_world_size(self.pg))]
        dist.all_gather(out, t, group=self.pg)
        return out

    def _broadcast(self, t, src: int):
        dist = self._dist()
        if dist is not None:
            dist.broadcast(t, src=src, group=self.pg)
        return t

    def _rank(self):
        dist = self._dist()
        return 0 if dist is None else dist.get_rank(self.pg)

    def _owner_of(self, w: int, ranges):
        for r, (a, b) in enumerate(ranges):
            if a <= w < b:
                return r
        raise ValueError(w)

    # ---- Algorithm 4's share ----
    def global_bests(self):
        """Per sharing group: (global index, f-hat) of the best incumbent
        over all ranks (smallest f-hat per point, lowest index on ties)."""
        C, deg, fhat = self.b.pools()
        fh = fhat.detach().to("cpu", torch.float64).numpy()
        nk = len(self.keys)
        loc = torch.full((nk, 2), float("inf"), dtype=torch.float64)
        for i, w in enumerate(range(self.w0, self.w1)):
            key = self.key_of[w]
            f = float(fh[i])
            cur_f, cur_w = float(loc[key, 0]), float(loc[key, 1])
            if f < cur_f or (f == cur_f and w < cur_w):
                loc[key, 0] = f
                loc[key, 1] = float(w)
        gathered = self._all_gather(loc.to(self.device))
        best = []
        for key in range(nk):
            bf, bw = float("inf"), float("inf")
            for t in gathered:
                f, w = float(t[key, 0]), float(t[key, 1])
                if f < bf or (f == bf and w < bw):
                    bf, bw = f, w
            best.append((int(bw), bf))
        return best

    def share_bases(self, ranges):
        """The cooperative base of every sharing group, broadcast from the
        rank that holds it: {key: (C k x d float32, deg k uint8)}."""
        C, deg, _ = self.b.pools()
        me = self._rank()
        out = {}
        for key, (wb, _) in enumerate(self.global_bests()):
            kk = self.keys[key][1]
            owner = self._owner_of(wb, ranges)
            if owner == me:
                i = wb - self.w0
                cb = C[self.C_off[i]: self.C_off[i] + kk * self.d].clone()
                db = deg[self.K_off[i]: self.K_off[i] + kk].clone()
            else:
                cb = torch.empty(kk * self.d, dtype=torch.float32, device=C.device)
                db = torch.empty(kk, dtype=torch.uint8, device=deg.device)
            # gloo and NCCL take float tensors; the flags travel as floats
            db_f = db.to(torch.float32)
            self._broadcast(cb, owner)
            self._broadcast(db_f, owner)
            out[key] = (cb, db_f.to(torch.uint8))
        return out

    def round(self, strategy: int, seed: int, rnd: int, ranges, n_competitive: int = 0):
        """One round of every local worker (Algorithms 3-5)."""
        coop = strategy == COOPERATIVE or (strategy == HYBRID and rnd >= n_competitive)
        if not coop:
            if self.w1 > self.w0:
                self.b.run_round(seed, rnd)
            return
        bases = self.share_bases(ranges)
        if self.w1 == self.w0:
            return
        C, deg, _ = self.b.pools()
        keep_C, keep_deg = C.clone(), deg.clone()
        for i, w in enumerate(range(self.w0, self.w1)):
            cb, db = bases[self.key_of[w]]
            kk = int(self.k[w])
            C[self.C_off[i]: self.C_off[i] + kk * self.d] = cb
            deg[self.K_off[i]: self.K_off[i] + kk] = db
        self.b.run_round(seed, rnd)
        acc = self.b.accepted()
        for i, w in enumerate(range(self.w0, self.w1)):
            if acc[i]:
                continue
            kk = int(self.k[w])
            a, b = self.C_off[i], self.C_off[i] + kk * self.d
            C[a:b] = keep_C[a:b]
            a, b = self.K_off[i], self.K_off[i] + kk
            deg[a:b] = keep_deg[a:b]

    # ---- Eq. 1 over row shards ----
    def objective(self, X_rows, C, deg):
        """Eq. 1 over all rows: this rank's block of rows, then one
        all-reduce of the FP64 partials."""
        f = self.b.objective(X_rows, C, deg).reshape(1).to(torch.float64)
        dist = self._dist()
        if dist is not None:
            f = f.to(self.device)
            dist.all_reduce(f, group=self.pg)
        return f

    def best(self, ranges, key: int = 0):
        """The best incumbent of sharing group `key` over all ranks:
        (global index, f-hat, C, deg)."""
        wb, fb = self.global_bests()[key]
        C, deg = self.share_bases(ranges)[key]
        return wb, fb, C, deg


class LibraryBackend:
    """The CUDA library as the compute of one rank: a batch of the rank's
    workers (worker0 = their first global index) on X."""

    def __init__(self, ctx, X, batch):
        from . import hpclust as H
        self.H = H
        self.ctx, self.X, self.batch = ctx, X, batch

    def pools(self):
        return self.batch.C, self.batch.degenerate, self.batch.fhat

    def offsets(self):
        return self.batch.C_off, self.batch.K_off

    def run_round(self, seed: int, rnd: int):
        self.H.hpc_round(self.ctx, self.X, self.batch, self.H.HPC_COMPETITIVE, seed, rnd)

    def accepted(self):
        return self.batch.accepted.cpu().numpy().astype(bool)

    def objective(self, rows, C, deg):
        return self.H.hpc_objective(self.ctx, rows, C, deg)
