"""Pins of the cost-model oracle (``oracle/costmodel.py``) against facts that
do not come from it: a network worked by hand, torch's float64 autograd,
central finite differences, Adam's closed forms, and a fit to a target the
network represents exactly.  A dropped term, a wrong sign, a transposed
weight matrix or a missing ReLU mask in the oracle fails one of them."""
import numpy as np
import pytest

from oracle import costmodel as cm


def _rand_params(rng, f=cm.F, h=cm.H, scale=0.3):
    return rng.normal(0.0, scale, cm.nparams(f, h))


def test_layout_size():
    assert cm.P == 1377 == cm.nparams()
    W1, b1, W2, b2, w3, b3 = cm.unpack(np.arange(cm.P, dtype=np.float64))
    assert W1.shape == (32, 8) and W1[0, 1] == 1 and W1[1, 0] == 8
    assert b1[0] == 256 and W2[0, 0] == 288 and W2[0, 1] == 289 and W2[1, 0] == 320
    assert b2[0] == 1312 and w3[0] == 1344 and b3 == 1376


def test_hand_worked_network():
    """F = 2, H = 2, two samples, every value worked by hand:
    x = (3, 1):  z1 = (2, 2.5), h1 = (2, 2.5), z2 = (2.5, 0.5), y = 3.75
    x = (-1, 2): z1 = (-3, 2.5), h1 = (0, 2.5), z2 = (0.5, 2.5), y = -6.25
    t = (3, -6): residuals (0.75, -0.25), loss = (0.5625 + 0.0625) / 2."""
    W1 = [[1.0, -1.0], [0.5, 2.0]]
    b1 = [0.0, -1.0]
    W2 = [[1.0, 0.0], [-1.0, 1.0]]
    b2 = [0.5, 0.0]
    w3 = [2.0, -3.0]
    b3 = 0.25
    p = np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]])
    X = np.array([[3.0, 1.0], [-1.0, 2.0]])
    t = np.array([3.0, -6.0])
    y = cm.predict(p, X, 2, 2)
    assert np.array_equal(y, [3.75, -6.25])
    loss, g = cm.loss_grad(p, X, t, 2, 2)
    assert loss == 0.3125
    # dL/dy = 2 r / N = (0.75, -0.25); worked through both layers by hand
    expect = np.concatenate([
        [11.25, 3.75, -7.5, -0.75],     # W1: sample 1 (3.75, -2.25) x (3, 1) + sample 2 (0, 0.75) x (-1, 2)
        [3.75, -1.5],                   # b1
        [3.0, 2.5, -4.5, -3.75],        # W2: (1.5, -2.25) x (2, 2.5) + (-0.5, 0.75) x (0, 2.5)
        [1.0, -1.5],                    # b2
        [1.75, -0.25],                  # w3: 0.75 (2.5, 0.5) - 0.25 (0.5, 2.5)
        [0.5],                          # b3
    ])
    assert np.array_equal(g, expect)


def test_against_torch_autograd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    for N in (1, 5, 300):
        p = _rand_params(rng)
        X = rng.normal(0.0, 1.0, (N, cm.F))
        t = rng.normal(0.0, 1.0, N)
        loss, g = cm.loss_grad(p, X, t)
        pt = torch.tensor(p, dtype=torch.float64, requires_grad=True)
        o = 0
        parts = []
        for shape in [(32, 8), (32,), (32, 32), (32,), (32,), ()]:
            size = int(np.prod(shape)) if shape else 1
            parts.append(pt[o:o + size].reshape(shape))
            o += size
        W1, b1, W2, b2, w3, b3 = parts
        Xt = torch.tensor(X)
        y = torch.relu(torch.relu(Xt @ W1.T + b1) @ W2.T + b2) @ w3 + b3
        L = torch.mean((y - torch.tensor(t)) ** 2)
        L.backward()
        assert loss == pytest.approx(L.item(), rel=1e-12)
        np.testing.assert_allclose(g, pt.grad.numpy(), rtol=1e-10, atol=1e-13)


def test_finite_differences():
    rng = np.random.default_rng(11)
    p = _rand_params(rng)
    X = rng.normal(0.0, 1.0, (40, cm.F))
    t = rng.normal(0.0, 1.0, 40)
    _, g = cm.loss_grad(p, X, t)
    h = 1e-6
    for i in list(range(0, cm.P, 37)) + [cm.P - 1, 256, 288, 1312, 1344]:
        e = np.zeros(cm.P)
        e[i] = h
        fd = (cm.loss_grad(p + e, X, t)[0] - cm.loss_grad(p - e, X, t)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8), i


def test_dead_units_get_no_gradient():
    """A hidden unit whose input is negative on every sample passes none."""
    rng = np.random.default_rng(3)
    p = _rand_params(rng)
    W1, b1, W2, b2, w3, b3 = cm.unpack(p.copy())
    p2 = p.copy()
    # unit 5 of layer 1: zero weights, negative bias
    p2[5 * 8:6 * 8] = 0.0
    p2[256 + 5] = -1.0
    X = rng.normal(0.0, 1.0, (20, cm.F))
    t = rng.normal(0.0, 1.0, 20)
    _, g = cm.loss_grad(p2, X, t)
    assert np.all(g[5 * 8:6 * 8] == 0.0) and g[256 + 5] == 0.0
    assert np.all(g[288 + 5:288 + 1024:32] == 0.0)  # column 5 of W2


def test_adam_first_step_closed_form():
    """From zero moments the bias-corrected step is lr g / (|g| + eps)."""
    rng = np.random.default_rng(5)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    g[3] = 0.0
    lr = 1e-3
    p1, m1, v1 = cm.adam_step(p, np.zeros(50), np.zeros(50), g, 1, lr)
    np.testing.assert_allclose(p1, p - lr * g / (np.abs(g) + cm.EPS), rtol=0, atol=1e-15)
    assert p1[3] == p[3]
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-12)


def test_adam_constant_gradient_keeps_its_step():
    """With a constant gradient m_hat = g and v_hat = g^2 at every step, so
    T steps move p by T lr g / (|g| + eps)."""
    rng = np.random.default_rng(6)
    p0 = rng.normal(size=20)
    g = rng.normal(size=20)
    p, m, v = p0, np.zeros(20), np.zeros(20)
    lr, T = 1e-2, 25
    for t in range(1, T + 1):
        p, m, v = cm.adam_step(p, m, v, g, t, lr)
    np.testing.assert_allclose(p, p0 - T * lr * g / (np.abs(g) + cm.EPS), rtol=0, atol=1e-11)


def test_training_fits_a_representable_target():
    """Targets made by a teacher network of the same shape: the loss of a
    student started near the teacher goes to (nearly) zero."""
    rng = np.random.default_rng(9)
    teacher = _rand_params(rng, scale=0.4)
    X = rng.normal(0.0, 1.0, (200, cm.F))
    t = cm.predict(teacher, X)
    student = teacher + rng.normal(0.0, 0.05, cm.P)
    p, m, v, losses = cm.train(student, X, t, 1500, 2e-3)
    assert losses[0] > 1e-3
    assert cm.loss_grad(p, X, t)[0] < 1e-3 * losses[0]


def test_train_resumes_exactly():
    """Training in two halves with the moments carried equals one run."""
    rng = np.random.default_rng(10)
    p0 = _rand_params(rng)
    X = rng.normal(0.0, 1.0, (30, cm.F))
    t = rng.normal(0.0, 1.0, 30)
    pa, ma, va, la = cm.train(p0, X, t, 20, 1e-3)
    pb, mb, vb, lb = cm.train(p0, X, t, 8, 1e-3)
    pc, mc, vc, lc = cm.train(pb, X, t, 12, 1e-3, mb, vb, 8)
    assert np.array_equal(pa, pc) and np.array_equal(la, np.concatenate([lb, lc]))
