"""Parity at the full sizes of the measured workloads, through the same calls
bench.py times: the plain FP32 workload (10^7 x 16), the precision workload
(2 x 10^7 x 128, k = 100), the batching workload (5 x 10^7 x 32, 64 workers)
and the large workload (2 x 10^8 x 64, k = 500, 51 GB on the device; CUDA-core
and wide TF32 searches).

At these sizes the oracle checks what it can compute one by one -- sampled
rows of the full-data objective, sampled workers of a full-size round -- and
properties that hold at any size check the rest:
  * every label is a nearest centroid (oracle, on the sampled rows; all rows
    for the 10^7-row workload);
  * the objective equals the double-precision sum of the squared distances
    of all rows to their labelled centroids, within 1e-6 relative (the bound
    of the FP32 direct-form distances it adds);
  * a sampled worker's round (sample draw, K-means++, Lloyd) matches the
    oracle's replay of that worker: objective within 1e-6, centroids per
    coordinate within 1e-6 relative plus 1e-9 of the largest coordinate.
"""
import numpy as np
import pytest
import torch

import oracle as orc
from lloyd_replay import RTOL, TIE, assert_centroids, check_parted_run
from paper_2311_04517_gb300 import hpclust as H
from paper_2311_04517_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = H.Context(0)
    yield c
    c.close()


def near_means(wl, k, seed):
    """Centroids close to the mixture means (a converged-looking solution)."""
    mu, sd, _ = synth.mixture_params(wl)
    rng = np.random.default_rng(seed)
    M = mu.numpy()[np.arange(k) % mu.shape[0]]     # k > components: several per mean
    C = M + 0.05 * rng.standard_normal((k, wl.d))
    return C.astype(np.float32)


def fp64_objective(X, C, labels, chunk=4_000_000):
    """sum_i ||x_i - c_{label_i}||^2 in double precision on the device."""
    Cd = C.double()
    tot = 0.0
    for a in range(0, X.shape[0], chunk):
        b = min(X.shape[0], a + chunk)
        diff = X[a:b].double() - Cd[labels[a:b].long()]
        tot += float((diff * diff).sum())
    return tot


def check_labels(lab_g, Xs, C, deg=None, what=""):
    lab_o, d1, d2, _ = orc.assign(Xs, C, deg)
    diff = np.flatnonzero(lab_g != lab_o)
    if diff.size:
        near = (d2[diff] - d1[diff]) <= TIE * d1[diff]
        assert near.all(), f"{what}: {np.count_nonzero(~near)} labels differ away from ties"
    return lab_o


def objective_case(ctx, wl, X, k, rows, seed):
    C = near_means(wl, k, seed)
    Cd = torch.from_numpy(C).cuda()
    labels = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    f = H.hpc_objective(ctx, X, Cd, labels_out=labels)
    ctx.check_status()
    f = float(f.item())
    assert f == pytest.approx(fp64_objective(X, Cd, labels), rel=RTOL)
    lab = labels.cpu().numpy()
    assert lab.min() >= 0 and lab.max() < k
    if rows is None:                      # every row through the oracle
        lab_o = check_labels(lab, X.cpu().numpy(), C, what=f"{wl.name} all rows")
        f_o = orc.objective(X.cpu().numpy(), C)
        assert f == pytest.approx(f_o, rel=RTOL)
    else:
        idx = np.sort(np.random.default_rng(seed).choice(X.shape[0], rows, replace=False))
        check_labels(lab[idx], X[torch.from_numpy(idx).cuda()].cpu().numpy(), C,
                     what=f"{wl.name} sampled rows")


def test_fp32_workload_objective_every_row(ctx):
    wl = synth.WORKLOADS["fp32"]
    X = synth.make_data(wl, "cuda")
    objective_case(ctx, wl, X, 25, None, 1)


def test_precision_workload_objective(ctx):
    wl = synth.WORKLOADS["precision"]
    X = synth.make_data(wl, "cuda")
    objective_case(ctx, wl, X, 100, 20_000, 2)   # TF32 tensor-core search (d = 128)
    del X
    torch.cuda.empty_cache()


@pytest.mark.parametrize("k", [25, 100])
def test_batching_workload_objective(ctx, k):
    # k = 25: split-TF32 tensor-core search; k = 100: CUDA-core search
    wl = synth.WORKLOADS["batching"]
    X = synth.make_data(wl, "cuda")
    objective_case(ctx, wl, X, k, 20_000, 3 + k)
    del X
    torch.cuda.empty_cache()


@pytest.mark.parametrize("form", [H.HPC_SEARCH_SIMT, H.HPC_SEARCH_TF32, H.HPC_SEARCH_SPLIT_BF16])
def test_large_workload_objective(ctx, form):
    # k = 500: the CUDA-core search (built-in choice) and the wide TF32 search
    # (four warpgroups over a tile's 512 accumulator columns)
    wl = synth.WORKLOADS["large"]
    X = synth.make_data(wl, "cuda")               # 2e8 x 64 float32, 51 GB
    ctx.set_objective_form(wl.d, 500, form)
    try:
        objective_case(ctx, wl, X, 500, 5_000, 4)
    finally:
        ctx.set_objective_form(wl.d, 500, -1)
    del X
    torch.cuda.empty_cache()


def oracle_worker(X, wl, ws, w, seed, rnd, host_X=None):
    """The oracle's replay of worker w's round from the all-degenerate start:
    its sample (indices from the oracle's Philox stream, rows gathered from
    X), K-means++ and Lloyd.  Returns (sample, K-means++ result, Lloyd run)."""
    s, k = int(ws.s[w]), int(ws.k[w])
    if host_X is not None:
        S, _ = orc.draw_sample(host_X, seed, w, rnd, s)
    else:
        idx = orc.sample_indices(X.shape[0], seed, w, rnd, s)
        S = X[torch.from_numpy(idx).cuda()].cpu().numpy()
    kp = orc.kmeanspp(S, np.zeros((k, wl.d), np.float32), np.ones(k, np.uint8), 3, seed, w, rnd)
    return S, kp, orc.lloyd(S, kp["C"], kp["degenerate"])


def check_worker(ctx, replay, batch, w, f_new, iters, what=""):
    """Worker w of a round against the oracle's replay.  When the two Lloyd
    runs part (another number of updates, or centroids off), the first
    difference must be a near tie (lock-step replay from the K-means++ start
    with the context's current search forms)."""
    S, kp, lo = replay
    C, deg = batch.centroids(w)
    g = dict(C=C.cpu().numpy(), degenerate=deg.cpu().numpy(), f=float(f_new[w]),
             iters=int(iters[w]))
    try:
        assert g["iters"] == lo["iters"]
        np.testing.assert_array_equal(g["degenerate"], lo["degenerate"])
        assert g["f"] == pytest.approx(lo["f"], rel=RTOL)
        assert_centroids(g["C"], lo["C"], f"{what} worker {w}")
    except AssertionError:
        check_parted_run(ctx, S, kp["C"], kp["degenerate"], g, lo)


def replay_worker(ctx, X, wl, ws, batch, w, seed, rnd, f_new, iters, host_X=None):
    replay = oracle_worker(X, wl, ws, w, seed, rnd, host_X)
    check_worker(ctx, replay, batch, w, f_new, iters)
    return replay[2]


def test_large_workload_round_sampled_workers(ctx):
    # one full-size round of the large workload: 128 workers, k = 500,
    # d = 64, samples of 65,536 to 1,048,576 rows drawn from 2e8 rows; the
    # Lloyd sums of k x d = 32,000 coordinates exceed a block's shared memory,
    # so every block adds into the global fixed-point sums.  The workers with
    # the smallest and the largest sample are replayed by the oracle from the
    # same all-degenerate start.
    wl = synth.WORKLOADS["large"]
    ws = synth.worker_setup(wl)
    X = synth.make_data(wl, "cuda")               # 2e8 x 64 float32, 51 GB
    seed, rnd = wl.seed, 0
    picks = (int(np.argmin(ws.s)), int(np.argmax(ws.s)))
    replays = {w: oracle_worker(X, wl, ws, w, seed, rnd) for w in picks}
    # both Lloyd searches: the CUDA cores (global fixed-point sums) and the
    # split-BF16 tensor cores (incremental sums of the rows that moved)
    for mode, form in ((0, "simt"), (2, "split_bf16")):
        ctx.set_tensor_cores(mode)
        try:
            sched = ctx.lloyd_schedule(int(ws.s.max()), wl.d, 500)
            assert not sched["smem_sums"] and sched["form"] == form, sched
            batch = H.Batch(wl.d, ws.s, ws.k, ws.group)
            H.hpc_round(ctx, X, batch, H.HPC_COMPETITIVE, seed, rnd)
            ctx.check_status()
            f_new = batch.f_new.cpu().numpy()
            iters = batch.iters.cpu().numpy()
            assert np.isfinite(f_new).all() and (iters >= 1).all()
            # every worker's incumbent was replaced (the start is +inf)
            assert batch.accepted.cpu().numpy().all()
            for w in picks:
                check_worker(ctx, replays[w], batch, w, f_new, iters, form)
        finally:
            ctx.set_tensor_cores(2)
        del batch
    del X
    torch.cuda.empty_cache()


def test_batching_workload_round_sampled_workers(ctx):
    # one full-size round of all 64 workers (one batched launch per phase);
    # three workers (k = 10, 25, 50) are replayed by the oracle from the
    # same all-degenerate start
    wl = synth.WORKLOADS["batching"]
    ws = synth.worker_setup(wl)
    X = synth.make_data(wl, "cuda")
    batch = H.Batch(wl.d, ws.s, ws.k, ws.group)
    seed, rnd = wl.seed, 0
    H.hpc_round(ctx, X, batch, H.HPC_COMPETITIVE, seed, rnd)
    ctx.check_status()
    f_new = batch.f_new.cpu().numpy()
    iters = batch.iters.cpu().numpy()
    Xh = X.cpu().numpy()
    for kk in (10, 25, 50, 100):
        cand = [w for w in range(wl.W) if int(ws.k[w]) == kk]
        w = min(cand, key=lambda v: int(ws.s[v]))        # the smallest sample of that k
        replay_worker(ctx, X, wl, ws, batch, w, seed, rnd, f_new, iters, host_X=Xh)
    del X
    torch.cuda.empty_cache()
