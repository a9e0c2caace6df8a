"""The search-form cost model on the GPU: forward pass, gradient and Adam
steps of the library's kernels against the FP64 oracle (``oracle/costmodel``),
determinism and exact resumption of training, the network inputs the library
builds, the guided autotuner, and what the trained network gains over the
search without it (on the measured GB300 sweep shipped with the package).

Tolerances.  The kernels compute in FP32: per-sample dot products of at most
32 terms, then sums over N samples in a fixed order, so each gradient entry
carries a relative error of about (32 + N) 2^-24 of the sum of its terms'
magnitudes.  The bars below (1e-4 of the largest entry for gradients, 1e-5
relative for losses and predictions) hold that bound with a wide margin for
the sizes tested and are far below the size of any dropped term or sign.
"""
import json
import math

import numpy as np
import pytest
import torch

import oracle as orc
from oracle import costmodel as ocm
from paper_2311_04517_gb300 import costmodel as cmod
from paper_2311_04517_gb300 import hpclust as H

pytestmark = pytest.mark.gpu
NP = H.HPC_CM_NPARAM
NF = H.HPC_CM_NFEAT


@pytest.fixture()
def ctx():
    c = H.Context(0)
    yield c
    c.close()


def _problem(N, seed, scale=0.3):
    g = np.random.default_rng(seed)
    p = g.normal(0.0, scale, NP).astype(np.float32)
    X = g.normal(0.0, 1.0, (N, NF)).astype(np.float32)
    t = g.normal(0.0, 1.0, N).astype(np.float32)
    return p, X, t


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda:0")


@pytest.mark.parametrize("N", [1, 63, 64, 65, 300, 1000])
def test_loss_grad_matches_oracle(ctx, N):
    p, X, t = _problem(N, 100 + N)
    loss, grad = H.hpc_costmodel_loss_grad(ctx, _dev(p), _dev(X), _dev(t))
    l_o, g_o = ocm.loss_grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert float(loss.item()) == pytest.approx(l_o, rel=1e-5)
    g = grad.cpu().numpy().astype(np.float64)
    scale = np.max(np.abs(g_o))
    assert np.max(np.abs(g - g_o)) <= 1e-4 * scale, np.max(np.abs(g - g_o)) / scale
    # exact zeros (dead units) stay exact zeros
    assert np.all(g[g_o == 0.0] == 0.0)


def test_predict_matches_oracle(ctx):
    p, X, _ = _problem(777, 5)
    y = H.hpc_costmodel_predict(ctx, _dev(p), _dev(X)).cpu().numpy()
    y_o = ocm.predict(p.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(y, y_o, rtol=1e-5, atol=1e-5 * np.max(np.abs(y_o)))


def test_one_adam_step_matches_oracle(ctx):
    p, X, t = _problem(200, 9)
    g = np.random.default_rng(19)
    m = g.normal(0.0, 0.01, NP).astype(np.float32)
    v = g.uniform(1e-4, 1e-3, NP).astype(np.float32)
    pd, md, vd = _dev(p), _dev(m), _dev(v)
    lr, step0 = 1e-3, 5
    losses = torch.empty(1, dtype=torch.float32, device="cuda:0")
    H.hpc_costmodel_train(ctx, pd, md, vd, _dev(X), _dev(t), 1, step0, lr, losses)
    P64 = [a.astype(np.float64) for a in (p, X, t, m, v)]
    l_o, g_o = ocm.loss_grad(P64[0], P64[1], P64[2])
    p_o, m_o, v_o = ocm.adam_step(P64[0], P64[3], P64[4], g_o, step0 + 1, lr)
    assert float(losses[0]) == pytest.approx(l_o, rel=1e-5)
    np.testing.assert_allclose(md.cpu().numpy(), m_o, rtol=0, atol=1e-4 * np.max(np.abs(m_o)))
    np.testing.assert_allclose(vd.cpu().numpy(), v_o, rtol=1e-4, atol=0)
    # an update is at most lr / sqrt(1 - beta2^t) * |m_hat| / sqrt(v_hat): the
    # gradient's FP32 error moves it by well under 1e-2 lr
    np.testing.assert_allclose(pd.cpu().numpy(), p_o, rtol=0, atol=1e-2 * lr)


def test_training_follows_the_oracle(ctx):
    """A student network fitted to a teacher of the same shape: the loss of
    every step agrees with the FP64 oracle run from the same start."""
    g = np.random.default_rng(21)
    teacher = g.normal(0.0, 0.4, NP)
    X = g.normal(0.0, 1.0, (500, NF)).astype(np.float32)
    t = ocm.predict(teacher, X.astype(np.float64)).astype(np.float32)
    p0 = (teacher + g.normal(0.0, 0.05, NP)).astype(np.float32)
    steps, lr = 300, 2e-3
    pd = _dev(p0)
    md = torch.zeros(NP, device="cuda:0")
    vd = torch.zeros(NP, device="cuda:0")
    losses = torch.empty(steps, dtype=torch.float32, device="cuda:0")
    H.hpc_costmodel_train(ctx, pd, md, vd, _dev(X), _dev(t), steps, 0, lr, losses)
    _, _, _, l_o = ocm.train(p0.astype(np.float64), X.astype(np.float64), t.astype(np.float64),
                             steps, lr)
    l = losses.cpu().numpy().astype(np.float64)
    assert l[-1] < 0.05 * l[0]
    rel = np.abs(l - l_o) / l_o
    assert np.max(rel) < 1e-2, (np.max(rel), int(np.argmax(rel)))


def test_training_is_deterministic_and_resumes_exactly(ctx):
    p, X, t = _problem(300, 33)
    Xd, td = _dev(X), _dev(t)

    def run(splits):
        pd, md, vd = _dev(p), torch.zeros(NP, device="cuda:0"), torch.zeros(NP, device="cuda:0")
        done = 0
        for s in splits:
            H.hpc_costmodel_train(ctx, pd, md, vd, Xd, td, s, done, 1e-3)
            done += s
        return pd.cpu().numpy(), md.cpu().numpy(), vd.cpu().numpy()

    a = run([20])
    b = run([20])
    c = run([8, 12])
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y) and np.array_equal(x, z)


def test_bad_arguments(ctx):
    p, X, t = _problem(4, 1)
    pd, Xd = _dev(p), _dev(X)
    m = torch.zeros(NP, device="cuda:0")
    for N in (0,):
        with pytest.raises(H.HPCError):
            H.hpc_costmodel_loss_grad(ctx, pd, Xd[:N], torch.empty(0, device="cuda:0"))
    with pytest.raises(H.HPCError):
        H.hpc_costmodel_train(ctx, pd, m, m.clone(), Xd, _dev(t), 1, 0, -1.0)
    with pytest.raises(H.HPCError):
        H.hpc_costmodel_train(ctx, pd, m, m.clone(), Xd, _dev(t), 1, 0, float("nan"))
    rc = ctx.lib.hpc_costmodel_train(ctx.h, H._ptr(pd), H._ptr(m), H._ptr(m), H._ptr(Xd),
                                     H._ptr(_dev(t)), 4, -1, 0, 1e-3, None)
    assert rc == H.HPC_ERR_ARG


def _separation(C, deg):
    live = [i for i in range(C.shape[0]) if not deg[i]]
    if len(live) < 2:
        return 0.0
    c = C[live].astype(np.float64)
    cmax2 = np.max(np.sum(c * c, axis=1))
    diff = c[:, None, :] - c[None, :, :]
    q = np.sum(diff * diff, axis=2)
    minsep = np.min(q[np.triu_indices(len(live), 1)])
    if minsep == 0.0:
        return 1.0
    return min(max(math.log2(cmax2 / minsep), 0.0), 40.0) / 40.0


@pytest.mark.parametrize("d,k", [(16, 25), (32, 100), (64, 500), (128, 200), (128, 300), (7, 9)])
def test_features(ctx, d, k):
    g = np.random.default_rng(d * 1000 + k)
    C = g.normal(0.0, 3.0, (k, d)).astype(np.float32)
    deg = (g.uniform(size=k) < 0.2).astype(np.uint8)
    feats, sup = H.hpc_costmodel_features(ctx, _dev(C), _dev(deg))
    feats = feats.numpy()
    cols = next(c for c in (32, 64, 128, 256, 512, 1 << 30) if k <= c)
    sep = _separation(C, deg)
    for f in range(3):
        row = feats[f]
        assert row[0] == pytest.approx(math.log2(d) / 7, rel=1e-6)
        assert row[1] == pytest.approx(math.log2(k) / 9, rel=1e-6)
        assert row[2] == pytest.approx(cols / k - 1, rel=1e-6)
        assert row[3] == pytest.approx(sep, rel=1e-5, abs=1e-6)
        assert list(row[4:7]) == [1.0 if q == f else 0.0 for q in range(3)]
        assert row[7] == (1.0 if k > 128 else 0.0)
    # the forms the library accepts for (d, k)
    for f in range(3):
        rc = ctx.lib.hpc_set_objective_form(ctx.h, d, k, f)
        assert (rc == H.HPC_OK) == bool(sup[f])
    ctx.set_objective_form(d, k, -1)


def test_features_degenerate_cases(ctx):
    C = np.zeros((4, 16), dtype=np.float32)
    C[0, 0] = 1.0
    C[1, 0] = 1.0       # coincides with centroid 0
    C[2, 3] = 5.0
    feats, _ = H.hpc_costmodel_features(ctx, _dev(C))
    assert feats[0, 3] == 1.0
    deg = np.array([0, 1, 1, 1], dtype=np.uint8)  # one live centroid
    feats, _ = H.hpc_costmodel_features(ctx, _dev(C), _dev(deg))
    assert feats[0, 3] == 0.0


def _trained_or_init():
    if cmod.OUT.exists():
        return np.asarray(json.loads(cmod.OUT.read_text())["params"], dtype=np.float32)
    return cmod.init_params(0, 0.0)


def test_guided_autotune_live(ctx):
    g = torch.Generator(device="cuda:0").manual_seed(3)
    n, d, k = 1 << 21, 16, 25
    mu = torch.rand((k, d), generator=g, device="cuda:0") * 20 - 10
    X = (mu[torch.randint(0, k, (n,), generator=g, device="cuda:0")]
         + torch.randn((n, d), generator=g, device="cuda:0")).contiguous()
    C = (mu + 0.1).contiguous()
    params = _dev(_trained_or_init())
    nsup = 3  # d = 16, k = 25: all three forms are built
    form, ms, timed = ctx.autotune_objective_guided(X, C, params, reps=2, margin=0.0)
    assert timed == 1 and len(ms) == 1 and form in (0, 1, 2)
    assert ctx.objective_form(n, d, k) == form
    form, ms, timed = ctx.autotune_objective_guided(X, C, params, reps=2, margin=1e30)
    assert timed == nsup and len(ms) == nsup
    # the fastest, or the built-in form within 1% of it
    assert ms[H.SEARCH_NAMES[form]] <= 1.01 * min(ms.values())
    assert ctx.objective_form(n, d, k) == form
    # the objective under the chosen form still matches the oracle's
    Xs = X[:200_000].contiguous()
    f = float(H.hpc_objective(ctx, Xs, C).item())
    assert f == pytest.approx(orc.objective(Xs.cpu().numpy(), C.cpu().numpy()), rel=1e-6)
    ctx.set_objective_form(d, k, -1)


def test_guided_autotune_rejects_bad_margin(ctx):
    X = torch.zeros((1024, 16), device="cuda:0")
    C = torch.zeros((4, 16), device="cuda:0")
    params = _dev(cmod.init_params(0))
    for margin in (-1.0, float("nan")):
        with pytest.raises(H.HPCError):
            ctx.autotune_objective_guided(X, C, params, margin=margin)


@pytest.mark.skipif(not cmod.OUT.exists(), reason="no measured sweep shipped")
def test_trained_network_gains_over_the_unguided_search(ctx):
    """Trains the network on the GPU from the measured sweep (the cluster
    counts in HOLDOUT_K held out), checks the gradient at the trained
    parameters against the oracle on the real training set, and replays the
    guided search on the held-out shapes: it must time fewer forms than the
    exhaustive search and pick a form within 5% of the fastest at least as
    often as the built-in table does."""
    data = json.loads(cmod.OUT.read_text())
    records = data["records"]
    train_r, held = cmod.split(records)
    feats, targets, _ = cmod.dataset(train_r)
    steps = data["train"]["steps"]
    params, losses = cmod.train(ctx, feats, targets, steps=steps)
    l = losses.cpu().numpy()
    assert l[-1] < 0.1 * l[0]
    # the shipped parameters came from this same training
    np.testing.assert_allclose(params.cpu().numpy(), np.asarray(data["params"], np.float32),
                               rtol=1e-3, atol=1e-3)
    # gradient parity on the real data at the trained parameters
    loss, grad = H.hpc_costmodel_loss_grad(ctx, params, _dev(feats), _dev(targets))
    p64 = params.cpu().numpy().astype(np.float64)
    l_o, g_o = ocm.loss_grad(p64, feats.astype(np.float64), targets.astype(np.float64))
    assert float(loss.item()) == pytest.approx(l_o, rel=1e-4)
    g = grad.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(g - g_o)) <= 1e-3 * np.max(np.abs(g_o))
    ev = cmod.evaluate(held, cmod.predict_records(ctx, params, held))
    assert ev["cases"] >= 10
    assert ev["guided_forms_timed"] < ev["exhaustive_forms_timed"]
    assert ev["guided_within_5pct"] >= ev["builtin_within_5pct"]
    assert ev["guided_within_5pct"] >= 0.75


def test_guided_autotune_refuses_a_nonfinite_network(ctx):
    X = torch.randn((4096, 16), device="cuda:0")
    C = torch.randn((8, 16), device="cuda:0")
    params = torch.full((NP,), float("nan"), device="cuda:0")
    with pytest.raises(H.HPCError):
        ctx.autotune_objective_guided(X, C, params)
    # the form table is untouched
    ctx.set_objective_form(16, 8, -1)


def test_guided_autotune_single_form(ctx):
    """d = 8: only the CUDA-core form is built, so exactly one is timed."""
    X = torch.randn((1 << 16, 8), device="cuda:0")
    C = torch.randn((12, 8), device="cuda:0")
    params = _dev(_trained_or_init())
    form, ms, timed = ctx.autotune_objective_guided(X, C, params, reps=1)
    assert form == H.HPC_SEARCH_SIMT and timed == 1 and list(ms) == ["simt"]
    feats, sup = H.hpc_costmodel_features(ctx, C)
    assert sup == [1, 0, 0]
    ctx.set_objective_form(8, 12, -1)
