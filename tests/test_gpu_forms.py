"""Search-form control of the full-data objective: every form the library
builds for a shape (CUDA cores, split TF32, TF32, split BF16) against the CPU oracle,
the per-shape form table (hpc_set_objective_form) and the measured choice
(hpc_autotune_objective).

Bars as for the other searches: labels equal the oracle's except near ties
(two nearest FP64 distances within 1e-6 relative); objectives within 1e-6
relative; every form agrees with the others on every label away from ties.
"""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_2311_04517_gb300 import hpclust as H

pytestmark = pytest.mark.gpu
RTOL = 1e-6
FORMS = (H.HPC_SEARCH_SIMT, H.HPC_SEARCH_SPLIT_TF32, H.HPC_SEARCH_TF32, H.HPC_SEARCH_SPLIT_BF16)


@pytest.fixture()
def ctx():
    c = H.Context(0)
    yield c
    c.close()


def mixture(n, d, comps, seed, spread=10.0, sd=1.0):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-spread, spread, (comps, d))
    z = rng.integers(0, comps, n)
    return (mu[z] + sd * rng.standard_normal((n, d))).astype(np.float32)


def built(d, k):
    ok = [H.HPC_SEARCH_SIMT]
    if d in (16, 32) and k <= 128:
        ok.append(H.HPC_SEARCH_SPLIT_TF32)
    if (d in (16, 32, 64) and k <= 512) or (d == 128 and k <= 256):
        ok.append(H.HPC_SEARCH_TF32)
    if (d == 64 and k <= 512) or (d == 128 and k <= 256):
        ok.append(H.HPC_SEARCH_SPLIT_BF16)
    return ok


def objective(ctx, X, C, deg=None):
    lab = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    f = H.hpc_objective(ctx, X, C, deg, labels_out=lab)
    ctx.check_status()
    return float(f.item()), lab.cpu().numpy()


@pytest.mark.parametrize("n,d,k", [(100037, 16, 25), (40001, 16, 33), (20000, 16, 128),
                                   (77777, 32, 25), (30000, 32, 100), (129, 32, 7),
                                   (20000, 64, 30), (8191, 128, 20),
                                   # wide TF32 search (k > 128): one or two TMEM banks per tile
                                   (30011, 16, 129), (20000, 16, 512), (25000, 32, 300),
                                   (40009, 64, 500), (12345, 64, 256), (300, 64, 200),
                                   (10007, 128, 256), (4097, 128, 131)])
def test_every_form_matches_oracle(ctx, n, d, k):
    # centroids near random rows: several per cluster, so that many rows sit
    # inside the TF32 error window and take the exact stages
    Xh = mixture(n, d, max(2, k // 2), seed=n + k, sd=1.5)
    rng = np.random.default_rng(k)
    Ch = (Xh[rng.choice(n, k, replace=n < k)] + 0.2 * rng.standard_normal((k, d))).astype(np.float32)
    deg = np.zeros(k, np.uint8)
    if k >= 8:
        deg[[1, k - 2]] = 1
    lab_o, d1, d2, f_o = orc.assign(Xh, Ch, deg)
    away = (d2 - d1) > 1e-6 * d1
    X, C, D = (torch.from_numpy(a).cuda() for a in (Xh, Ch, deg))
    forms = built(d, k)
    for form in forms:
        ctx.set_objective_form(d, k, form)
        assert ctx.objective_form(n, d, k) == form
        f, lab = objective(ctx, X, C, D)
        assert f == pytest.approx(f_o, rel=RTOL), H.SEARCH_NAMES[form]
        np.testing.assert_array_equal(lab[away], lab_o[away], err_msg=H.SEARCH_NAMES[form])


def test_form_table_and_modes(ctx):
    n, d, k = 1000, 16, 25
    default = ctx.objective_form(n, d, k)
    assert default == H.HPC_SEARCH_SIMT          # built-in choice at d = 16
    ctx.set_objective_form(d, k, H.HPC_SEARCH_TF32)
    assert ctx.objective_form(n, d, k) == H.HPC_SEARCH_TF32
    assert ctx.objective_form(n, d, 26) == default   # another shape is untouched
    ctx.set_tensor_cores(0)                          # mode 0 overrides the table
    assert ctx.objective_form(n, d, k) == H.HPC_SEARCH_SIMT
    ctx.set_tensor_cores(1)
    assert ctx.objective_form(n, d, k) == H.HPC_SEARCH_SPLIT_TF32
    ctx.set_tensor_cores(2)
    ctx.set_objective_form(d, k, -1)
    assert ctx.objective_form(n, d, k) == default
    # forms that are not built for a shape are refused
    with pytest.raises(H.HPCError) as e:
        ctx.set_objective_form(8, 25, H.HPC_SEARCH_SPLIT_TF32)
    assert e.value.code == H.HPC_ERR_UNSUPPORTED
    with pytest.raises(H.HPCError) as e:
        ctx.set_objective_form(64, 513, H.HPC_SEARCH_TF32)
    assert e.value.code == H.HPC_ERR_UNSUPPORTED
    with pytest.raises(H.HPCError) as e:
        ctx.set_objective_form(128, 257, H.HPC_SEARCH_TF32)
    assert e.value.code == H.HPC_ERR_UNSUPPORTED
    ctx.set_objective_form(64, 200, H.HPC_SEARCH_TF32)    # the wide search
    assert ctx.objective_form(n, 64, 200) == H.HPC_SEARCH_TF32
    with pytest.raises(H.HPCError) as e:
        ctx.set_objective_form(16, 25, 7)
    assert e.value.code == H.HPC_ERR_ARG


@pytest.mark.parametrize("d,k", [(16, 25), (32, 50), (64, 100), (8, 10), (64, 300)])
def test_autotune_picks_a_built_form_and_keeps_results(ctx, d, k):
    n = 400_000
    Xh = mixture(n, d, k, seed=d + k, sd=1.0)
    rng = np.random.default_rng(d)
    X = torch.from_numpy(Xh).cuda()
    C = torch.from_numpy(Xh[rng.choice(n, k, replace=False)]).cuda()
    ctx.set_tensor_cores(0)
    f0, lab0 = objective(ctx, X, C)
    ctx.set_tensor_cores(2)
    form, ms = ctx.autotune_objective(X, C, reps=3)
    forms = built(d, k)
    assert form in forms
    assert sorted(ms) == sorted(H.SEARCH_NAMES[f] for f in forms)
    assert all(t > 0 for t in ms.values())
    # the fastest, or the built-in form within 1% of it
    assert ms[H.SEARCH_NAMES[form]] <= 1.01 * min(ms.values())
    assert ctx.objective_form(n, d, k) == form
    f1, lab1 = objective(ctx, X, C)
    assert f1 == pytest.approx(f0, rel=1e-9)
    Xs = Xh[:20000]
    lab_o, d1, d2, _ = orc.assign(Xs, C.cpu().numpy())
    away = (d2 - d1) > 1e-6 * d1
    np.testing.assert_array_equal(lab1[:20000][away], lab_o[away])
    np.testing.assert_array_equal(lab1[:20000][away], lab0[:20000][away])


def test_autotune_argument_errors(ctx):
    X = torch.zeros((1000, 16), device="cuda")
    C = torch.zeros((5, 16), device="cuda")
    with pytest.raises(H.HPCError):
        ctx.autotune_objective(X, C, reps=0)
    with pytest.raises(H.HPCError):
        ctx.autotune_objective(X[:0], C)


def test_wide_search_edge_cases(ctx):
    # k > 128 on the wide TF32 search: no live centroid, a non-finite row,
    # degenerate slots in both TMEM banks, a ragged last tile, determinism
    d, k = 64, 300
    ctx.set_objective_form(d, k, H.HPC_SEARCH_TF32)
    C = torch.from_numpy(mixture(k, d, 20, 5)).cuda()
    X = torch.ones((300, d), device="cuda")
    H.hpc_objective(ctx, X, C, torch.ones(k, dtype=torch.uint8, device="cuda"))
    assert ctx.sync_status() == H.HPC_ERR_DEGENERATE_ALL
    Xn = mixture(1000, d, 20, 6)
    Xn[777, 5] = np.inf
    H.hpc_objective(ctx, torch.from_numpy(Xn).cuda(), C)
    assert ctx.sync_status() == H.HPC_ERR_NONFINITE
    Xh = mixture(50_001, d, 40, 7, sd=2.0)
    Ch = (Xh[np.random.default_rng(7).choice(50_001, k, replace=False)]).astype(np.float32)
    deg = np.zeros(k, np.uint8)
    deg[[0, 100, 255, 256, 299]] = 1
    lab_o, d1, d2, f_o = orc.assign(Xh, Ch, deg)
    X, C, D = (torch.from_numpy(a).cuda() for a in (Xh, Ch, deg))
    fa, la = objective(ctx, X, C, D)
    fb, lb = objective(ctx, X, C, D)
    assert fa == fb
    np.testing.assert_array_equal(la, lb)
    assert fa == pytest.approx(f_o, rel=RTOL)
    away = (d2 - d1) > 1e-6 * d1
    np.testing.assert_array_equal(la[away], lab_o[away])
    assert not np.isin(la, [0, 100, 255, 256, 299]).any()
