"""The pieces of a multi-GPU job on one GPU, through the C ABI:
  * worker0: a batch split into two batches (the second with worker0 = its
    first global index) runs exactly the rounds of one batch of all workers;
  * the cooperative share as the multi-rank driver does it (write the best
    incumbent over the workers' slots, run the competitive round, restore the
    incumbents that were not replaced) equals the device-side cooperative
    round, bit for bit, and both match the oracle's cooperative round;
  * the row-block objective plus a sum equals the whole objective."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_2311_04517_gb300 import hpclust as H
from paper_2311_04517_gb300 import multirank as MR

pytestmark = pytest.mark.gpu

S = [3000, 4500, 2000, 3500, 2500, 4000]
K = [6, 6, 9, 6, 9, 6]
G = [0, 0, 1, 0, 1, 0]
D = 16


@pytest.fixture(scope="module")
def ctx():
    c = H.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def data():
    rng = np.random.default_rng(61)
    mu = rng.uniform(-10, 10, (10, D))
    z = rng.integers(0, 10, 40000)
    Xh = (mu[z] + 1.3 * rng.standard_normal((40000, D))).astype(np.float32)
    return Xh, torch.from_numpy(Xh).cuda()


def same(a, b):
    for x, y in ((a.C, b.C), (a.degenerate, b.degenerate), (a.fhat, b.fhat)):
        assert torch.equal(x, y)


def test_split_batches_equal_one_batch(ctx, data):
    _, X = data
    whole = H.Batch(D, S, K, G)
    lo = H.Batch(D, S[:3], K[:3], G[:3])
    hi = H.Batch(D, S[3:], K[3:], G[3:], worker0=3)
    for r in range(3):
        H.hpc_round(ctx, X, whole, H.HPC_COMPETITIVE, 7, r)
        H.hpc_round(ctx, X, lo, H.HPC_COMPETITIVE, 7, r)
        H.hpc_round(ctx, X, hi, H.HPC_COMPETITIVE, 7, r)
    ctx.check_status()
    for w in range(len(S)):
        part, i = (lo, w) if w < 3 else (hi, w - 3)
        Cw, dw = whole.centroids(w)
        Cp, dp = part.centroids(i)
        assert torch.equal(Cw, Cp) and torch.equal(dw, dp)
        assert float(whole.fhat[w]) == float(part.fhat[i])


@pytest.mark.parametrize("strategy", [H.HPC_COOPERATIVE, H.HPC_HYBRID])
def test_driver_share_equals_device_share(ctx, data, strategy):
    Xh, X = data
    native = H.Batch(D, S, K, G, n_competitive=2)
    split = H.Batch(D, S, K, G, n_competitive=2)
    job = MR.RankedRun(MR.LibraryBackend(ctx, X, split), S, K, G, D, 0, len(S),
                       device=torch.device("cuda"))
    ranges = MR.worker_ranges(S, K, 1)
    st = orc.RoundState(D, S, K, G)
    for r in range(4):
        H.hpc_round(ctx, X, native, strategy, 5, r)
        job.round(strategy, 5, r, ranges, n_competitive=2)
        orc.round_(Xh, st, strategy, 5, r, n_competitive=2)
        ctx.check_status()
        same(native, split)
        for w in range(len(S)):
            C, deg = split.centroids(w)
            Co, dego = st.centroids(w)
            np.testing.assert_array_equal(deg.cpu().numpy(), dego)
            tol = 1e-6 * np.abs(Co) + 1e-9 * max(1.0, float(np.abs(Co).max()))
            assert (np.abs(C.cpu().numpy().astype(np.float64) - Co) <= tol).all()
        np.testing.assert_allclose(split.fhat.cpu().numpy(), st.fhat, rtol=1e-6)


def test_row_block_objective(ctx, data):
    Xh, X = data
    C = X[:12].clone()
    whole = float(H.hpc_objective(ctx, X, C).item())
    parts = 0.0
    for r in range(3):
        a, b = MR.row_range(X.shape[0], 3, r)
        parts += float(H.hpc_objective(ctx, X[a:b], C).item())
    ctx.check_status()
    # row blocks regroup the rows each thread adds (FP32 sums of a few rows
    # before the pair), about 1e-9 of the total; the contract is 1e-6
    assert parts == pytest.approx(whole, rel=1e-8)
    assert whole == pytest.approx(orc.objective(Xh, Xh[:12]), rel=1e-6)
