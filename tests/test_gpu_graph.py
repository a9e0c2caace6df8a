"""A prepared round (hpc_round_prepare / hpc_round_enqueue) gives the same
results as hpc_round, enqueued directly and replayed from a CUDA graph that
recorded one round: the round index comes from a device counter that each
round advances, so one recorded round serves every round (bit-exact
centroids, objectives, iteration counts and decisions)."""
import numpy as np
import pytest
import torch

from paper_2311_04517_gb300 import hpclust as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = H.Context(0)
    yield c
    c.close()


def mixture(n, d, comps, seed, sd=1.0):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-10, 10, (comps, d))
    z = rng.integers(0, comps, n)
    return torch.from_numpy((mu[z] + sd * rng.standard_normal((n, d))).astype(np.float32)).cuda()


SETUP = dict(s=[3000, 4500, 2000, 3500, 2500], k=[6, 6, 9, 6, 9], group=[0, 0, 1, 0, 1])


def same(a: H.Batch, b: H.Batch):
    assert torch.equal(a.C, b.C)
    assert torch.equal(a.degenerate, b.degenerate)
    assert torch.equal(a.fhat, b.fhat)
    assert torch.equal(a.f_new, b.f_new)
    assert torch.equal(a.iters, b.iters)
    assert torch.equal(a.accepted, b.accepted)


@pytest.mark.parametrize("strategy", [H.HPC_COMPETITIVE, H.HPC_COOPERATIVE, H.HPC_HYBRID])
def test_prepared_round_matches_hpc_round(ctx, strategy):
    X = mixture(40000, 16, 10, 51, sd=1.3)
    ref = H.Batch(16, n_competitive=2, **SETUP)
    prep = H.Batch(16, n_competitive=2, **SETUP)
    H.hpc_round_prepare(ctx, X, prep, strategy, 11, 0)
    for r in range(5):
        H.hpc_round(ctx, X, ref, strategy, 11, r)
        H.hpc_round_enqueue(ctx)
        ctx.check_status()
        same(ref, prep)


@pytest.mark.parametrize("strategy", [H.HPC_COOPERATIVE, H.HPC_HYBRID])
def test_prepared_round_replays_from_a_cuda_graph(ctx, strategy):
    X = mixture(40000, 16, 10, 52, sd=1.3)
    ref = H.Batch(16, n_competitive=2, **SETUP)
    gb = H.Batch(16, n_competitive=2, **SETUP)
    R = 5
    for r in range(R):
        H.hpc_round(ctx, X, ref, strategy, 13, r)
    ctx.check_status()
    H.hpc_round_prepare(ctx, X, gb, strategy, 13, 0)
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    old = ctx.stream if hasattr(ctx, "stream") else torch.cuda.current_stream()
    try:
        with torch.cuda.graph(g, stream=side):
            ctx.set_stream(side)
            H.hpc_round_enqueue(ctx)      # recorded, not run
        for _ in range(R):
            g.replay()
        torch.cuda.synchronize()
    finally:
        ctx.set_stream(old if isinstance(old, torch.cuda.Stream) else torch.cuda.current_stream())
    ctx.check_status()
    same(ref, gb)


def test_round_arguments_are_checked(ctx):
    X = mixture(1000, 8, 3, 7)
    b = H.Batch(8, [100, 100], [3, 3])
    with pytest.raises(H.HPCError):
        H.hpc_round(ctx, X, b, 7, 0, 0)                       # unknown strategy
    with pytest.raises(H.HPCError):
        H.hpc_round(ctx, X, b, H.HPC_COMPETITIVE, 0, 0, max_iter=100_001)
    with pytest.raises(H.HPCError):
        H.hpc_round(ctx, X, b, H.HPC_COMPETITIVE, 0, 0, n_candidates=9)
    with pytest.raises(H.HPCError):
        H.hpc_round(ctx, X, H.Batch(8, [0, 100], [3, 3]), H.HPC_COMPETITIVE, 0, 0)  # s = 0
    fresh = H.Context(0)
    try:
        with pytest.raises(H.HPCError):
            H.hpc_round_enqueue(fresh)                         # nothing prepared
    finally:
        fresh.close()
    ctx.check_status()


def test_readme_example_runs(ctx):
    from paper_2311_04517_gb300 import synth
    X = synth.make_data("tiny", "cuda")
    batch = H.Batch(2, s=[2000] * 4, k=[5] * 4)
    for r in range(3):
        H.hpc_round(ctx, X, batch, H.HPC_COMPETITIVE, seed=0, round_=r)
    best = int(torch.argmin(batch.fhat))
    C, deg = batch.centroids(best)
    labels = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    f = H.hpc_objective(ctx, X, C, deg, labels_out=labels)
    ctx.check_status()
    assert float(f.item()) > 0 and int(labels.max()) < 5
