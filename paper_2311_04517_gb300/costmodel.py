"""Measured data, training and evaluation of the search-form cost model.

The library's network (``hpc_costmodel_*`` in include/hpclust.h) predicts
ln(ns per row) of each search form of the full-data objective (Eq. 1) from
inputs the library builds.  This module

* ``sweep``: measures every built form on synthetic Gaussian mixtures over a
  grid of (d, k) and two spreads, with incumbent centroids from the
  library's own K-means++ and Lloyd on a sample (so that near ties between
  centroids look like the ones the objective meets in a run), recording the
  library's network inputs, the measured times and the built-in choice;
* ``train``: fits the network on the GPU with the library's training kernels
  (full-batch Adam from a seeded He initialisation);
* ``evaluate``: replays the guided search of
  ``hpc_autotune_objective_guided`` on recorded times -- rank the built forms
  by predicted time, time the best-ranked one and each other one predicted
  within a factor (1 + margin) -- and counts the forms timed and how often
  the chosen form is within 5% of the fastest, beside the exhaustive search
  (every form timed) and the built-in table (none timed).

``python -m paper_2311_04517_gb300.costmodel`` runs all three on cuda:0 and
writes ``costmodel_gb300.json`` next to this file: the records, the trained
parameters and the held-out evaluation.  Held out are the cluster counts in
HOLDOUT_K, which the network never sees in training.
"""
from __future__ import annotations

import dataclasses
import json
import math
import sys
import time
from pathlib import Path

import numpy as np
import torch

from . import hpclust as H
from . import synth

OUT = Path(__file__).resolve().parent / "costmodel_gb300.json"
DIMS = (16, 32, 64, 128)
KS = (10, 16, 25, 32, 50, 64, 100, 128, 200, 256, 500)
HOLDOUT_K = (16, 64, 200)
SPREADS = {
    # well separated components: few rows near a tie
    "separated": (("uniform", -20.0, 20.0), ("uniform", 0.5, 2.0)),
    # overlapping components: many rows near a tie
    "overlapping": (("normal", 2.0), ("const", 1.0)),
}
SAMPLE = 65_536
LLOYD_ITERS = 30
REPS = 3
MARGIN = 0.25


def rows_for(d: int) -> int:
    """Timing rows: at least 256 MB of X, more than the 129 MB L2."""
    return (1 << 22) if d <= 32 else (1 << 21)


def _incumbents(ctx, X, k, seed):
    """Centroids a worker would hold: greedy K-means++ then Lloyd on a sample."""
    d = X.shape[1]
    S = torch.empty((SAMPLE, d), dtype=torch.float32, device=X.device)
    H.hpc_draw_sample(ctx, X, seed, 0, 0, SAMPLE, S_out=S)
    C = torch.zeros((k, d), dtype=torch.float32, device=X.device)
    deg = torch.ones(k, dtype=torch.uint8, device=X.device)
    H.hpc_kmeanspp(ctx, S, C, deg, seed=seed, worker=0, round_=0)
    H.hpc_lloyd(ctx, S, C, deg, max_iter=LLOYD_ITERS)
    return C, deg


def sweep(ctx, dims=DIMS, ks=KS, spreads=tuple(SPREADS), seed: int = 1, log=print):
    records = []
    dev = ctx.device
    for spread in spreads:
        means, sd = SPREADS[spread]
        for d in dims:
            n = rows_for(d)
            for k in ks:
                if d == 128 and k > 256:
                    continue  # only the CUDA-core form is built there
                wl = dataclasses.replace(synth.WORKLOADS["fp32"], name=f"cm_{spread}", n=n, d=d,
                                         comps=k, means=means, sd=sd, weights="equal")
                X = synth.make_data(wl, device=dev, seed=seed + 1000 * d + k)
                C, deg = _incumbents(ctx, X, k, seed + k)
                feats, sup = H.hpc_costmodel_features(ctx, C, deg)
                if sum(sup) < 2:
                    continue  # one form: nothing to choose
                ctx.set_objective_form(d, k, -1)
                builtin = ctx.objective_form(n, d, k)
                form, ms = ctx.autotune_objective(X, C, deg, reps=REPS)
                ctx.set_objective_form(d, k, -1)
                rec = {"d": d, "k": k, "spread": spread, "n": n,
                       "features": [[float(v) for v in row] for row in feats.tolist()],
                       "supported": sup,
                       "ms": [float(ms.get(H.SEARCH_NAMES[f], -1.0)) for f in range(3)],
                       "builtin": builtin, "fastest": form}
                records.append(rec)
                log(f"d={d:4d} k={k:4d} {spread:11s} sep={feats[0, 3]:.3f} "
                    + " ".join(f"{H.SEARCH_NAMES[f]}={rec['ms'][f]:.3f}" for f in range(3)
                               if sup[f]))
                del X
    return records


def dataset(records):
    """Network inputs and targets ln(ns per row), one row per built form."""
    feats, targets, where = [], [], []
    for i, r in enumerate(records):
        for f in range(3):
            if r["supported"][f] and r["ms"][f] > 0:
                feats.append(r["features"][f])
                targets.append(math.log(r["ms"][f] * 1e6 / r["n"]))
                where.append((i, f))
    return (np.asarray(feats, dtype=np.float32), np.asarray(targets, dtype=np.float32), where)


def init_params(seed: int, target_mean: float = 0.0):
    """He-normal weights, zero biases, output bias at the mean target."""
    F, Hd = H.HPC_CM_NFEAT, H.HPC_CM_HIDDEN
    g = np.random.default_rng(seed)
    W1 = g.normal(0.0, math.sqrt(2.0 / F), (Hd, F))
    W2 = g.normal(0.0, math.sqrt(2.0 / Hd), (Hd, Hd))
    w3 = g.normal(0.0, math.sqrt(1.0 / Hd), Hd)
    p = np.concatenate([W1.ravel(), np.zeros(Hd), W2.ravel(), np.zeros(Hd), w3, [target_mean]])
    assert p.size == H.HPC_CM_NPARAM
    return p.astype(np.float32)


def train(ctx, feats, targets, steps: int = 4000, lr: float = 3e-3, seed: int = 0):
    """Full-batch Adam on the GPU; returns (params, losses) device tensors."""
    dev = ctx.device
    p = torch.tensor(init_params(seed, float(np.mean(targets))), device=dev)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    Xf = torch.tensor(feats, device=dev).contiguous()
    t = torch.tensor(targets, device=dev).contiguous()
    losses = torch.empty(steps, dtype=torch.float32, device=dev)
    H.hpc_costmodel_train(ctx, p, m, v, Xf, t, steps, 0, lr, losses)
    return p, losses


def guided_choice(pred, ms, supported, margin: float = MARGIN):
    """The guided search on recorded times, with the library's own plan
    (hpc_costmodel_plan): (chosen form, forms timed)."""
    order, timed_mask = H.hpc_costmodel_plan(pred, supported, margin)
    best, timed = None, 0
    for f, t in zip(order, timed_mask):
        if f < 0 or not t:
            continue
        timed += 1
        if best is None or ms[f] < ms[best]:
            best = f
    return best, timed


def evaluate(records, preds, margin: float = MARGIN):
    """Held-out comparison of the guided, exhaustive and built-in choices.
    preds[i][f]: predicted ln(ns per row) of form f for record i."""
    g_ok = b_ok = g_timed = e_timed = 0
    for r, pr in zip(records, preds):
        ms = r["ms"]
        fast = min(ms[f] for f in range(3) if r["supported"][f])
        f, timed = guided_choice(pr, ms, r["supported"], margin)
        g_ok += ms[f] <= 1.05 * fast
        g_timed += timed
        e_timed += sum(r["supported"])
        b_ok += ms[r["builtin"]] <= 1.05 * fast
    n = len(records)
    return {"cases": n, "margin": margin,
            "guided_within_5pct": g_ok / n, "guided_forms_timed": g_timed / n,
            "exhaustive_within_5pct": 1.0, "exhaustive_forms_timed": e_timed / n,
            "builtin_within_5pct": b_ok / n, "builtin_forms_timed": 0.0}


def predict_records(ctx, params, records):
    F = H.HPC_CM_NFEAT
    feats = torch.tensor([row for r in records for row in r["features"]],
                         dtype=torch.float32, device=ctx.device).view(-1, F).contiguous()
    y = H.hpc_costmodel_predict(ctx, params, feats).cpu().numpy()
    return y.reshape(len(records), 3).tolist()


def split(records, holdout_k=HOLDOUT_K):
    train_r = [r for r in records if r["k"] not in holdout_k]
    held = [r for r in records if r["k"] in holdout_k]
    return train_r, held


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="measure, train and evaluate the cost model")
    ap.add_argument("--out", default=str(OUT), help="where to write the JSON")
    args = ap.parse_args(argv)
    ctx = H.Context(0)
    t0 = time.time()
    records = sweep(ctx)
    t_sweep = time.time() - t0
    train_r, held = split(records)
    feats, targets, _ = dataset(train_r)
    params, losses = train(ctx, feats, targets)
    ev = evaluate(held, predict_records(ctx, params, held))
    ev_train = evaluate(train_r, predict_records(ctx, params, train_r))
    out = {"device": torch.cuda.get_device_name(0),
           "command": "python -m paper_2311_04517_gb300.costmodel",
           "timing": {"reps": REPS, "sample": SAMPLE, "lloyd_iters": LLOYD_ITERS,
                      "sweep_s": round(t_sweep, 1)},
           "holdout_k": list(HOLDOUT_K),
           "train": {"samples": int(len(targets)), "steps": int(losses.numel()), "lr": 3e-3,
                     "seed": 0, "loss_first": float(losses[0]), "loss_last": float(losses[-1])},
           "heldout": ev, "train_eval": ev_train,
           "params": [float(x) for x in params.cpu().tolist()],
           "records": records}
    Path(args.out).write_text(json.dumps(out, indent=1))
    print(json.dumps({k: out[k] for k in ("device", "timing", "train", "heldout", "train_eval")}))
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
