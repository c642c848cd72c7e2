"""Pins of the FP64 MLP reference: SiLU identities, a hand-computed network,
gradients against central differences of the loss, and one Adam step in
closed form."""
import numpy as np

from oracle import mlp as M


def test_silu_identities():
    a = np.linspace(-20, 20, 401)
    # (the tanh form cancels for large negative a, hence the absolute floor)
    np.testing.assert_allclose(M.silu(a), a * 0.5 * (1 + np.tanh(a / 2)), rtol=1e-14, atol=2e-15)
    e = 1e-6
    fd = (M.silu(a + e) - M.silu(a - e)) / (2 * e)
    np.testing.assert_allclose(M.silu_grad(a), fd, rtol=1e-8, atol=1e-10)
    assert M.silu(0.0) == 0.0 and abs(M.silu_grad(0.0) - 0.5) < 1e-16


def test_forward_hand_computed():
    W = [np.array([[1.0, -1.0]]), np.eye(2), np.eye(2), np.array([[2.0], [3.0]])]
    b = [np.array([0.5, 0.0]), np.zeros(2), np.zeros(2), np.array([1.0])]
    x = np.array([[1.0]])
    y, _ = M.forward(W, b, x)
    h = np.array([1.5, -1.0])
    for _ in range(3):
        h = h / (1 + np.exp(-h))
    assert abs(y[0, 0] - (2 * h[0] + 3 * h[1] + 1.0)) < 1e-15


def test_gradients_against_central_differences():
    rng = np.random.default_rng(0)
    sizes = [5, 7, 6, 7, 3]
    W, b = M.init(sizes, seed=1)
    x = rng.normal(size=(9, 5))
    t = rng.normal(size=(9, 3))
    y, cache = M.forward(W, b, x)
    gW, gb = M.backward(W, b, cache, y, t)
    e = 1e-6
    for l in range(4):
        for (i, j) in [(0, 0), (sizes[l] - 1, sizes[l + 1] - 1), (2, 1)]:
            W[l][i, j] += e
            lp = M.loss(M.forward(W, b, x)[0], t)
            W[l][i, j] -= 2 * e
            lm = M.loss(M.forward(W, b, x)[0], t)
            W[l][i, j] += e
            assert abs((lp - lm) / (2 * e) - gW[l][i, j]) < 1e-7 * max(1, abs(gW[l][i, j]))
        b[l][0] += e
        lp = M.loss(M.forward(W, b, x)[0], t)
        b[l][0] -= 2 * e
        lm = M.loss(M.forward(W, b, x)[0], t)
        b[l][0] += e
        assert abs((lp - lm) / (2 * e) - gb[l][0]) < 1e-7


def test_adam_first_step_closed_form():
    p = [np.array([1.0, -2.0, 0.5])]
    g = [np.array([0.3, -1e-3, 0.0])]
    opt = M.Adam(p, lr=0.01)
    opt.step(p, g)
    # bias-corrected m = g, v = g^2 -> step = lr g / (|g| + eps)
    want = np.array([1.0, -2.0, 0.5]) - 0.01 * g[0] / (np.abs(g[0]) + 1e-8)
    np.testing.assert_allclose(p[0], want, rtol=1e-15)


def test_training_reduces_loss():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(256, 4))
    t = np.stack([np.sin(x[:, 0]), x[:, 1] * x[:, 2]], axis=1)
    W, b = M.init([4, 16, 16, 16, 2], seed=3)
    opt = M.Adam(W + b, lr=3e-3)
    l0 = M.loss(M.forward(W, b, x)[0], t)
    for _ in range(200):
        y, c = M.forward(W, b, x)
        gW, gb = M.backward(W, b, c, y, t)
        opt.step(W + b, gW + gb)
    assert M.loss(M.forward(W, b, x)[0], t) < 0.2 * l0


def test_rounding_points_of_the_reduced_precision_mode():
    """With rnd, the input and every hidden activation are rounded before the
    next product and the output is not; the back-propagated gradient is
    rounded where the products read it and the bias gradient sums it
    unrounded.  A chain of one-unit layers makes each point visible."""
    q = lambda v: np.round(np.asarray(v) * 8.0) / 8.0        # a coarse rounding, step 1/8
    W = [np.array([[1.0]]), np.array([[1.0]]), np.array([[1.0]]), np.array([[3.0]])]
    b = [np.array([0.0]), np.array([0.0]), np.array([0.0]), np.array([0.01])]
    x = np.array([[1.3]])                                   # q(1.3) = 1.25
    y, (h, a) = M.forward(W, b, x, rnd=q)
    v = 1.25
    for _ in range(3):
        v = q(M.silu(v))
    assert abs(y[0, 0] - (3.0 * v + 0.01)) < 1e-15          # output unrounded
    assert h[0][0, 0] == 1.25 and all(hh[0, 0] == q(hh[0, 0]) for hh in h[1:4])
    t = np.array([[0.0]])
    gW, gb = M.backward(W, b, (h, a), y, t, rnd=q)
    g = 2.0 * y[0, 0]
    assert abs(gb[3][0] - g) < 1e-15                        # bias: unrounded
    assert abs(gW[3][0, 0] - h[3][0, 0] * q(g)) < 1e-15     # weight: rounded g
    yn, cn = M.forward(W, b, x)
    gWn, gbn = M.backward(W, b, cn, yn, t)
    assert abs(gbn[3][0] - 2.0 * yn[0, 0]) < 1e-15 and yn[0, 0] != y[0, 0]
