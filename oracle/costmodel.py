"""Cost-model oracle: the schedule-choice network in float64 with numpy.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: imported by
``tests/`` alone; the GPU library and its Python binding never import it,
and it shares no code with the CUDA kernels.

The paper has no learned component (Sections 3-4); this network serves the
one tile-schedule choice of the library that changes a kernel's speed
several-fold, the search form of the full-data objective (Eq. 1), and never
touches an assignment or an objective value.  It is a two-hidden-layer
perceptron with ReLU activations (Rumelhart, Hinton and Williams 1986, for
the gradient by back-propagation) trained on the mean squared error of the
log time per row with Adam (Kingma and Ba, ICLR 2015, Algorithm 1: moments
m and v, bias corrections 1 - beta^t, step lr * m_hat / (sqrt(v_hat) + eps)).

Flat parameter vector (the interface both sides read; each side has its own
code): W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3 -- F = 8 inputs,
H = 32 hidden units, 1377 values.

    y(x) = b3 + w3 . relu(b2 + W2 relu(b1 + W1 x))
    L    = (1/N) sum_i (y(x_i) - t_i)^2

Pins (``tests/test_oracle_costmodel.py``): a network worked by hand,
torch's float64 autograd for the loss and every gradient entry, central
finite differences, Adam's closed forms (first step = -lr sign(g); constant
gradient keeps that step), and training that fits a target the network can
represent exactly.
"""
from __future__ import annotations

import numpy as np

F = 8
H = 32
P = H * F + H + H * H + H + H + 1  # 1377

BETA1 = 0.9
BETA2 = 0.999
EPS = 1e-8


def unpack(p, f: int = F, h: int = H):
    """Views (W1, b1, W2, b2, w3, b3) of the flat vector p."""
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + h * f].reshape(h, f); o += h * f
    b1 = p[o:o + h]; o += h
    W2 = p[o:o + h * h].reshape(h, h); o += h * h
    b2 = p[o:o + h]; o += h
    w3 = p[o:o + h]; o += h
    b3 = p[o]; o += 1
    assert o == p.size, (o, p.size)
    return W1, b1, W2, b2, w3, b3


def nparams(f: int = F, h: int = H) -> int:
    return h * f + h + h * h + h + h + 1


def forward(p, X, f: int = F, h: int = H):
    """Predictions y (N) and the activations the gradient needs."""
    W1, b1, W2, b2, w3, b3 = unpack(p, f, h)
    X = np.asarray(X, dtype=np.float64).reshape(-1, f)
    z1 = X @ W1.T + b1            # N x H
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2           # N x H
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3              # N
    return y, (X, z1, h1, z2, h2)


def predict(p, X, f: int = F, h: int = H):
    return forward(p, X, f, h)[0]


def loss_grad(p, X, t, f: int = F, h: int = H):
    """Mean squared error and its gradient with respect to p (same layout).

    Back-propagation through the two layers: dL/dy_i = 2 (y_i - t_i) / N;
    the ReLU passes the gradient where its input is positive (a zero input
    passes none)."""
    W1, b1, W2, b2, w3, b3 = unpack(p, f, h)
    t = np.asarray(t, dtype=np.float64).reshape(-1)
    y, (X, z1, h1, z2, h2) = forward(p, X, f, h)
    N = y.size
    r = y - t
    loss = float(np.sum(r * r) / N)
    gy = 2.0 * r / N                          # N
    g_w3 = h2.T @ gy                          # H
    g_b3 = np.sum(gy)
    g_z2 = np.outer(gy, w3) * (z2 > 0.0)      # N x H
    g_W2 = g_z2.T @ h1                        # H x H
    g_b2 = g_z2.sum(axis=0)
    g_z1 = (g_z2 @ W2) * (z1 > 0.0)           # N x H
    g_W1 = g_z1.T @ X                         # H x F
    g_b1 = g_z1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, g


def adam_step(p, m, v, g, t: int, lr: float, beta1: float = BETA1, beta2: float = BETA2,
              eps: float = EPS):
    """One Adam update at step t (1-based); returns new (p, m, v)."""
    p = np.asarray(p, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def train(p0, X, t, steps: int, lr: float, m0=None, v0=None, t0: int = 0,
          f: int = F, h: int = H):
    """Full-batch Adam from p0; returns (p, m, v, losses), losses[s] being
    the loss at the parameters step s started from."""
    p = np.array(p0, dtype=np.float64)
    m = np.zeros_like(p) if m0 is None else np.array(m0, dtype=np.float64)
    v = np.zeros_like(p) if v0 is None else np.array(v0, dtype=np.float64)
    losses = []
    for s in range(steps):
        loss, g = loss_grad(p, X, t, f, h)
        losses.append(loss)
        p, m, v = adam_step(p, m, v, g, t0 + s + 1, lr)
    return p, m, v, np.array(losses)
