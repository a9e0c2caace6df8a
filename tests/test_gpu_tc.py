"""Tensor-core nearest-centroid searches against the CPU oracle and against
the SIMT search: split TF32 (three tcgen05 MMAs per K step, row operand in
tensor memory) for d = 16 / 32, TF32 with exact resolution for d = 64 / 128.

Bars: labels equal the oracle's except near ties (two nearest FP64 distances
within 1e-6 relative); objectives within 1e-6 relative; the two GPU forms
agree on every label away from ties.
"""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_2311_04517_gb300 import hpclust as H

pytestmark = pytest.mark.gpu
RTOL = 1e-6


@pytest.fixture(scope="module")
def ctx():
    c = H.Context(0)
    yield c
    c.set_tensor_cores(2)
    c.close()


def mixture(n, d, comps, seed, spread=10.0, sd=1.0):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-spread, spread, (comps, d))
    z = rng.integers(0, comps, n)
    return (mu[z] + sd * rng.standard_normal((n, d))).astype(np.float32)


def run(ctx, X, C, deg, tc):
    ctx.set_tensor_cores(int(tc))
    lab = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    f = H.hpc_objective(ctx, torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda(),
                        None if deg is None else torch.from_numpy(deg).cuda(), labels_out=lab)
    ctx.check_status()
    return float(f.item()), lab.cpu().numpy()


@pytest.mark.parametrize("n,d,k", [(127, 16, 25), (128, 16, 25), (100037, 16, 25), (5000, 16, 1),
                                   (40000, 16, 32), (40001, 16, 33), (30000, 16, 64),
                                   (20011, 16, 100), (20000, 16, 128), (77777, 32, 25),
                                   (50001, 32, 50), (30000, 32, 128), (129, 32, 7),
                                   (20000, 64, 30), (12345, 64, 100), (8191, 128, 20),
                                   (10000, 128, 128), (300, 128, 5)])
def test_tc_objective_matches_oracle_and_simt(ctx, n, d, k):
    X = mixture(n, d, max(2, k), seed=n + k, sd=1.5)
    rng = np.random.default_rng(k)
    C = (X[rng.choice(n, k, replace=n < k)] + 0.2 * rng.standard_normal((k, d))).astype(np.float32)
    deg = np.zeros(k, np.uint8)
    if k >= 8:
        deg[[2, k - 1]] = 1
    lab_o, d1, d2, f_o = orc.assign(X, C, deg)
    f_tc, lab_tc = run(ctx, X, C, deg, True)
    f_sm, lab_sm = run(ctx, X, C, deg, False)
    assert f_tc == pytest.approx(f_o, rel=RTOL)
    assert f_sm == pytest.approx(f_o, rel=RTOL)
    away = (d2 - d1) > 1e-6 * d1
    np.testing.assert_array_equal(lab_tc[away], lab_o[away])
    np.testing.assert_array_equal(lab_sm[away], lab_o[away])


def test_tc_near_ties_are_resolved_exactly(ctx):
    rng = np.random.default_rng(3)
    d = 16
    c0 = rng.uniform(50, 60, d)
    c1 = c0 + rng.uniform(-1, 1, d) * 0.5
    mid = (c0 + c1) / 2
    n = 8192
    X = (mid + rng.standard_normal((n, d)) * 1e-4
         + np.outer(rng.uniform(-1e-3, 1e-3, n), c1 - c0)).astype(np.float32)
    C = np.stack([c0, c1]).astype(np.float32)
    _, lab = run(ctx, X, C, None, True)
    lab_o, d1, d2, _ = orc.assign(X, C)
    strict = (d2 - d1) > 1e-12 * d1
    np.testing.assert_array_equal(lab[strict], lab_o[strict])


@pytest.mark.parametrize("d", [16, 32])
def test_tc_margins_across_the_error_window(ctx, d):
    # rows on a line through the bisector of two centroids, at distances
    # from it spread over 1e-5 .. 10: their top-2 margins span the split-TF32
    # error window on both sides
    rng = np.random.default_rng(d)
    c0 = rng.uniform(50, 60, d)
    c1 = c0 + rng.uniform(-1, 1, d) * 0.5
    far = c0 + 40.0
    mid = (c0 + c1) / 2
    u = (c1 - c0) / np.linalg.norm(c1 - c0)
    t = np.logspace(-5, 1, 4000)
    t = np.concatenate([t, -t])
    X = (mid + np.outer(t, u) + rng.standard_normal((t.size, d)) * 1e-6).astype(np.float32)
    C = np.stack([c0, far, c1]).astype(np.float32)
    _, lab = run(ctx, X, C, None, True)
    lab_o, d1, d2, f_o = orc.assign(X, C)
    away = (d2 - d1) > 1e-6 * d1
    np.testing.assert_array_equal(lab[away], lab_o[away])


def test_tc_tight_clusters_need_rescoring(ctx):
    # several centroids inside one cluster: many rows fall inside the TF32
    # error window and must be settled by the exact stages
    rng = np.random.default_rng(17)
    d, k = 32, 24
    X = mixture(30000, d, 4, 17, spread=20.0, sd=1.0)
    C = (X[rng.choice(30000, k, replace=False)] + 0.01 * rng.standard_normal((k, d))).astype(np.float32)
    lab_o, d1, d2, f_o = orc.assign(X, C)
    f_tc, lab_tc = run(ctx, X, C, None, True)
    assert f_tc == pytest.approx(f_o, rel=RTOL)
    away = (d2 - d1) > 1e-6 * d1
    np.testing.assert_array_equal(lab_tc[away], lab_o[away])


def test_tc_auto_policy_is_default(ctx):
    ctx.set_tensor_cores(2)
    X = mixture(5000, 64, 8, 3)
    C = X[:8].copy()
    f, lab = run(ctx, X, C, None, 2)
    lab_o, d1, d2, f_o = orc.assign(X, C)
    assert f == pytest.approx(f_o, rel=RTOL)


def test_tc_edge_cases(ctx):
    ctx.set_tensor_cores(True)
    C = torch.from_numpy(np.array([[0] * 16, [1] * 16], np.float32)).cuda()
    # no live centroid
    X = torch.ones((300, 16), device="cuda")
    H.hpc_objective(ctx, X, C, torch.ones(2, dtype=torch.uint8, device="cuda"))
    assert ctx.sync_status() == H.HPC_ERR_DEGENERATE_ALL
    # non-finite row
    Xn = np.ones((300, 16), np.float32)
    Xn[200, 3] = np.nan
    H.hpc_objective(ctx, torch.from_numpy(Xn).cuda(), C)
    assert ctx.sync_status() == H.HPC_ERR_NONFINITE
    # deterministic
    Xr = mixture(60000, 16, 25, 4)
    Cr = Xr[:25].copy()
    a, la = run(ctx, Xr, Cr, None, True)
    b, lb = run(ctx, Xr, Cr, None, True)
    assert a == b
    np.testing.assert_array_equal(la, lb)
