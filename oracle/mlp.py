"""FP64 reference of the step/guess predictor MLP (numpy).

TEST INFRASTRUCTURE ONLY: used by the tests and the benchmark's CPU leg to
check the CUDA forward/backward/Adam kernels.  Plain definitions, no fusion.

Network: x (d0) -> [Linear -> SiLU] x 3 (width H) -> Linear -> y (dout),
SiLU(a) = a * sigmoid(a).  Loss: mean squared error over batch and outputs.
Optimiser: Adam (Kingma & Ba) with bias correction.

Weights are stored as W[l] with shape (d_in, d_out) (y = x @ W + b).
"""
from __future__ import annotations

import numpy as np


def silu(a):
    return a / (1.0 + np.exp(-a))


def silu_grad(a):
    s = 1.0 / (1.0 + np.exp(-a))
    return s * (1.0 + a * (1.0 - s))


def init(sizes, seed=0):
    """He-style uniform init; sizes = [d0, H, H, H, dout]."""
    rng = np.random.default_rng(seed)
    W, b = [], []
    for din, dout in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / din)
        W.append(rng.uniform(-lim, lim, size=(din, dout)))
        b.append(np.zeros(dout))
    return W, b


def forward(W, b, x, rnd=None):
    """Returns (y, cache) with pre-activations a_l and activations h_l.

    rnd (optional) rounds every matrix the forward products read: the input
    and each hidden activation before it enters the next layer (a
    reduced-precision network that stores its activations at that
    precision; the caller rounds the weights).  The arithmetic stays FP64
    and the output is not rounded."""
    r = (lambda v: v) if rnd is None else rnd
    h = [r(np.asarray(x, dtype=np.float64))]
    a = []
    L = len(W)
    for l in range(L):
        z = h[-1] @ W[l] + b[l]
        a.append(z)
        h.append(r(silu(z)) if l < L - 1 else z)
    return h[-1], (h, a)


def loss(y, t):
    d = y - t
    return float(np.mean(d * d))


def backward(W, b, cache, y, t, rnd=None):
    """Gradients of the MSE loss w.r.t. every W[l], b[l].

    rnd (optional) rounds the back-propagated gradient where the products
    read it (the weight gradient and the gradient of the layer input); the
    bias gradient sums it unrounded."""
    r = (lambda v: v) if rnd is None else rnd
    h, a = cache
    L = len(W)
    g = 2.0 * (y - t) / y.size
    gW, gb = [None] * L, [None] * L
    for l in range(L - 1, -1, -1):
        if l < L - 1:
            g = g * silu_grad(a[l])
        gr = r(g)
        gW[l] = h[l].T @ gr
        gb[l] = g.sum(axis=0)
        g = gr @ W[l].T
    return gW, gb


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [np.zeros_like(p) for p in params]
        self.v = [np.zeros_like(p) for p in params]
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t
        for p, g, m, v in zip(params, grads, self.m, self.v):
            m *= self.b1
            m += (1.0 - self.b1) * g
            v *= self.b2
            v += (1.0 - self.b2) * g * g
            p -= self.lr * (m / c1) / (np.sqrt(v / c2) + self.eps)
