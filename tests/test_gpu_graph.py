"""A prepared round (hpc_round_prepare / hpc_round_enqueue) gives the same
results as hpc_round, enqueued directly and replayed from a CUDA graph that
recorded one round: the round index comes from a device counter that each
round advances, so one recorded round serves every round (bit-exact
centroids, objectives, iteration counts and decisions)."""
import numpy as np
import pytest
import torch

import oracle as orc
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


def assert_matches_oracle(batch, st, res):
    """The batch's state after a round against the oracle's (Algorithms 3-5):
    flags, iteration counts and decisions equal, objectives within 1e-6,
    centroids per coordinate within 1e-6 relative plus 1e-9 of the largest."""
    d = batch.d
    for w in range(batch.W):
        C, deg = batch.centroids(w)
        Co, dego = st.centroids(w)
        np.testing.assert_array_equal(deg.cpu().numpy(), dego)
        Co64 = Co.astype(np.float64)
        tol = 1e-6 * np.abs(Co64) + 1e-9 * max(1.0, float(np.abs(Co64).max()))
        assert (np.abs(C.cpu().numpy().astype(np.float64) - Co64) <= tol).all(), f"worker {w}"
    np.testing.assert_array_equal(batch.iters.cpu().numpy(), res["iters"])
    np.testing.assert_array_equal(batch.accepted.cpu().numpy().astype(bool), res["accepted"])
    np.testing.assert_allclose(batch.f_new.cpu().numpy(), res["f_new"], rtol=1e-6)
    np.testing.assert_allclose(batch.fhat.cpu().numpy(), st.fhat, rtol=1e-6)


@pytest.mark.parametrize("strategy", [H.HPC_COOPERATIVE, H.HPC_HYBRID])
def test_prepared_round_replays_from_a_cuda_graph(ctx, strategy):
    X = mixture(40000, 16, 10, 52, sd=1.3)
    Xh = X.cpu().numpy()
    ref = H.Batch(16, n_competitive=2, **SETUP)
    gb = H.Batch(16, n_competitive=2, **SETUP)
    st = orc.RoundState(16, SETUP["s"], SETUP["k"], SETUP["group"])
    R = 5
    for r in range(R):
        H.hpc_round(ctx, X, ref, strategy, 13, r)
    ctx.check_status()
    H.hpc_round_prepare(ctx, X, gb, strategy, 13, 0)
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    old = ctx.stream if hasattr(ctx, "stream") else torch.cuda.current_stream()
    try:
        ctx.set_phase_timing(True)
        with torch.cuda.graph(g, stream=side):
            ctx.set_stream(side)
            H.hpc_round_enqueue(ctx)      # recorded, not run
        for r in range(R):
            g.replay()
            # every replay times itself: the event records are graph nodes
            ms = ctx.phase_times()
            assert ms["sample"] > 0 and ms["kmeanspp"] > 0 and ms["lloyd"] > 0, ms
            # each replayed round against the oracle's round r, directly
            res = orc.round_(Xh, st, strategy, 13, r, n_competitive=2)
            torch.cuda.synchronize()
            assert_matches_oracle(gb, st, res)
        torch.cuda.synchronize()
    finally:
        ctx.set_phase_timing(False)
        ctx.set_stream(old if isinstance(old, torch.cuda.Stream) else torch.cuda.current_stream())
    ctx.check_status()
    same(ref, gb)


def test_phase_timing_of_issued_rounds(ctx):
    X = mixture(20000, 8, 6, 53)
    b = H.Batch(8, [3000, 2000], [5, 7])
    with pytest.raises(H.HPCError):
        ctx.phase_times()                 # nothing timed yet
    ctx.set_phase_timing(True)
    try:
        H.hpc_round(ctx, X, b, H.HPC_COMPETITIVE, 1, 0)
        ms = ctx.phase_times()
        assert all(v > 0 for v in ms.values()), ms
    finally:
        ctx.set_phase_timing(False)
    ctx.check_status()


def test_lloyd_schedule_reports_the_planned_launch(ctx):
    small = ctx.lloyd_schedule(100_000, 16, 25)
    assert small["smem_sums"] and small["blocks"] >= 1 and small["smem_bytes"] > 0
    big = ctx.lloyd_schedule(1_048_576, 64, 500)
    assert not big["smem_sums"]           # 500 x 64 x 8 bytes exceed a block's shared memory
    with pytest.raises(H.HPCError):
        ctx.lloyd_schedule(0, 16, 25)


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
