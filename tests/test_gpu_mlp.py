"""The step/guess predictor's CUDA kernels against the FP64 numpy reference
(oracle/mlp.py), entry by entry: forward values and loss gradients (FP32
check mode to 1e-5 of each block's scale; BF16 tensor-core mode within the
propagated BF16 rounding bound), an Adam step, the prediction entry point,
training progress, and the feature / target kernels that connect the
network to the integrator."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp as M  # noqa: E402
from paper_1607_03884_gb300 import kin, synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kin.lib()


def unpack(p, din, w, dout):
    sizes = [din, w, w, w, dout]
    W, b, q = [], [], 0
    for a, c in zip(sizes[:-1], sizes[1:]):
        W.append(p[q:q + a * c].reshape(a, c).astype(np.float64))
        q += a * c
        b.append(p[q:q + c].astype(np.float64))
        q += c
    assert q == p.size
    return W, b


def bf16(x):
    return torch.from_numpy(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


U_BF16 = 2.0 ** -8      # a BF16 rounding flip moves a value by at most 2^-8 of it


def U_ACC(K):
    """FP32 accumulation of K products (the standard K u bound, u = 2^-24), plus
    the fast exponential of SiLU, relative to the sum of the absolute terms."""
    return (K + 4) * 2.0 ** -24


def bf16_bounds(W, b, cache, y, t):
    """First-order element-wise bounds on |GPU - reference| for the BF16 mode.

    Both sides round the same FP32 values at the same points (input, hidden
    activations, back-propagated gradient); they differ by FP32 accumulation
    and, where a value lies near a rounding boundary, by one BF16 step of
    that value.  Those differences are propagated layer by layer through
    absolute-value products, with |silu'| <= 1.1 and |silu''| <= 0.5."""
    h, a = cache
    L = len(W)
    aW = [np.abs(w) for w in W]
    Eh = np.zeros_like(h[0])                                   # the input is rounded alike
    EC = []
    for l in range(L):
        E = Eh @ aW[l] + U_ACC(W[l].shape[0]) * (np.abs(h[l]) @ aW[l])
        EC.append(E)
        if l < L - 1:
            Eh = 1.1 * E + U_BF16 * np.abs(h[l + 1])
    Ey = EC[-1]
    g = 2.0 * (y - t) / y.size
    Eg = 2.0 * Ey / y.size
    EW, Eb = [None] * L, [None] * L
    hin_err = [np.zeros_like(h[0])] + [1.1 * EC[l] + U_BF16 * np.abs(h[l + 1])
                                       for l in range(L - 1)]
    for l in range(L - 1, -1, -1):
        if l < L - 1:
            sg = 1.1 * np.ones_like(a[l])
            Eg = Eg * sg + np.abs(g) * 0.5 * EC[l]
            g = g * M.silu_grad(a[l])
        Egr = Eg + U_BF16 * np.abs(g)
        nb = h[l].shape[0]
        EW[l] = (hin_err[l].T @ np.abs(g) + np.abs(h[l]).T @ Egr
                 + U_ACC(nb) * (np.abs(h[l]).T @ np.abs(g)))
        Eb[l] = Eg.sum(axis=0) + U_ACC(nb) * np.abs(g).sum(axis=0)
        dH = g @ W[l].T
        Eg = Egr @ aW[l].T + U_ACC(W[l].shape[1]) * (np.abs(g) @ aW[l].T)
        g = dH
    return Ey, EW, Eb


def flat(Ws, bs):
    return np.concatenate([np.concatenate([a.ravel(), c]) for a, c in zip(Ws, bs)])


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("din,w,dout,n", [(16, 64, 40, 77), (56, 32, 160, 130),
                                         (56, 256, 160, 4100)])
def test_forward_and_gradients_against_fp64_reference(precision, din, w, dout, n):
    """Every output and every gradient entry against the FP64 reference
    (4100 rows: the weight-gradient GEMMs split K over several CTAs).
    FP32 mode: |gpu - ref| <= 1e-5 (|ref| + the block's largest |ref|), block
    by block (each W_l, each b_l, the output).  BF16 mode: the reference
    rounds to BF16 where the kernels do, and each entry must lie within the
    propagated rounding bound of bf16_bounds."""
    rng = np.random.default_rng(din + w)
    net = kin.MLP(din, w, dout, precision=precision, seed=3)
    p = net.get_params()
    p[:] += rng.normal(0, 0.01, p.size).astype(np.float32)   # nonzero biases too
    net.set_params(p)
    X = rng.normal(size=(n, din)).astype(np.float32)
    T = rng.normal(size=(n, dout)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    Y = torch.empty((n, dout), dtype=torch.float32, device="cuda")
    net.forward(Xd, Y)
    g = torch.empty(net.num_params(), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    net.grad(Xd, Td, grad_out=g, loss_out=loss)
    W, b = unpack(p.astype(np.float64), din, w, dout)
    x = X.astype(np.float64)
    t = T.astype(np.float64)
    rnd = bf16 if precision == "bf16" else None
    if rnd is not None:
        W = [bf16(Wl) for Wl in W]
    y, cache = M.forward(W, b, x, rnd=rnd)
    gW, gb = M.backward(W, b, cache, y, t, rnd=rnd)
    yg = Y.cpu().numpy().astype(np.float64)
    gg = g.cpu().numpy().astype(np.float64)
    gWg, gbg = unpack(gg, din, w, dout)
    if precision == "fp32":
        def bound(ref):
            return 1e-5 * (np.abs(ref) + np.abs(ref).max())
        blocks = [("y", yg, y, bound(y))]
        blocks += [(f"W{l}", gWg[l], gW[l], bound(gW[l])) for l in range(4)]
        blocks += [(f"b{l}", gbg[l], gb[l], bound(gb[l])) for l in range(4)]
    else:
        Ey, EW, Eb = bf16_bounds(W, b, cache, y, t)
        blocks = [("y", yg, y, Ey + 1e-6 * np.abs(y))]
        blocks += [(f"W{l}", gWg[l], gW[l], EW[l] + 1e-6 * np.abs(gW[l])) for l in range(4)]
        blocks += [(f"b{l}", gbg[l], gb[l], Eb[l] + 1e-6 * np.abs(gb[l])) for l in range(4)]
    worst = {}
    for name, got, ref, bnd in blocks:
        assert got.shape == ref.shape, name
        ratio = np.abs(got - ref) / (bnd + 1e-30)
        worst[name] = float(ratio.max())
        assert np.all(np.abs(got - ref) <= bnd), (name, np.unravel_index(ratio.argmax(), ratio.shape),
                                                   worst[name])
    print(f"\n{precision} {din}x{w}x{dout} n={n}: largest |gpu - ref| / bound per block "
          + ", ".join(f"{k} {v:.2f}" for k, v in worst.items()))
    L0 = M.loss(y, t)
    assert abs(loss.item() - L0) <= (1e-5 if precision == "fp32" else 2e-2) * L0


def test_adam_step_against_the_reference():
    """One FP32-mode Adam step from zero moments: every parameter moves as the
    reference's Adam (bias-corrected, beta 0.9 / 0.999, eps 1e-8) moves it
    with the reference gradient."""
    rng = np.random.default_rng(8)
    din, w, dout, n = 12, 32, 10, 50
    net = kin.MLP(din, w, dout, precision="fp32", seed=4)
    p = net.get_params()
    p[:] += rng.normal(0, 0.01, p.size).astype(np.float32)
    net.set_params(p)
    X = rng.normal(size=(n, din)).astype(np.float32)
    T = rng.normal(size=(n, dout)).astype(np.float32)
    lr = 1e-3
    net.train_step(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), lr)
    torch.cuda.synchronize()
    p1 = net.get_params().astype(np.float64)
    W, b = unpack(p.astype(np.float64), din, w, dout)
    y, cache = M.forward(W, b, X.astype(np.float64))
    gW, gb = M.backward(W, b, cache, y, T.astype(np.float64))
    params = [q for pair in zip(W, b) for q in pair]
    grads = [q for pair in zip(gW, gb) for q in pair]
    opt = M.Adam(params, lr=lr)
    opt.step(params, grads)
    ref = flat(params[0::2], params[1::2])
    # the first step moves each parameter by lr g/(|g| + eps): about lr, sign of g
    gflat = flat(grads[0::2], grads[1::2])
    sig = np.abs(gflat) > 1e-4          # away from the eps-dominated tiny gradients
    np.testing.assert_allclose(p1[sig], ref[sig], rtol=0, atol=2e-3 * lr + 1e-6)
    assert np.all(np.abs(p1[~sig] - p.astype(np.float64)[~sig]) <= 1.01 * lr + 1e-6)


def test_training_reduces_loss_on_device():
    rng = np.random.default_rng(0)
    n, din, dout = 4096, 16, 40
    X = rng.normal(size=(n, din)).astype(np.float32)
    Wt = rng.normal(size=(din, dout)) / 4
    T = np.tanh(X @ Wt).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    net = kin.MLP(din, 64, dout, precision="bf16", seed=1)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    losses = []
    for it in range(300):
        i = (it * 512) % n
        net.train_step(Xd[i:i + 512], Td[i:i + 512], 2e-3, loss_out=loss)
        losses.append(loss.item())
    assert np.mean(losses[-20:]) < 0.1 * np.mean(losses[:5]), (losses[:5], losses[-5:])


def test_feature_target_and_prediction_kernels():
    mech = synth.make_mechanism("h2")
    st = synth.make_states(mech, 300, seed=4)
    ns, n = mech.ns, st.n
    Y, T, P = (torch.from_numpy(a).cuda() for a in (st.Y, st.T, st.P))
    X = torch.empty((n, 3 + ns), dtype=torch.float32, device="cuda")
    kin.features(ns, Y, T, P, 1e-4, X)
    want = np.concatenate([np.log(st.T)[:, None], np.log(st.P)[:, None],
                           np.full((n, 1), np.log(1e-4)),
                           np.log10(np.maximum(st.Y.T, 1e-12))], axis=1)
    np.testing.assert_allclose(X.cpu().numpy(), want, rtol=2e-6, atol=2e-6)
    mean = torch.empty(3 + ns, dtype=torch.float32, device="cuda")
    std = torch.empty_like(mean)
    kin.moments(X, mean, std)
    np.testing.assert_allclose(mean.cpu().numpy(), want.mean(0), rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(std.cpu().numpy(), np.maximum(want.std(0), 1e-12), rtol=1e-4, atol=1e-6)
    h = torch.from_numpy(np.linspace(1e-9, 1e-6, n)).cuda()
    z = torch.from_numpy(np.arange(3 * ns * n, dtype=np.float64).reshape(3 * ns, n)).cuda()
    tg = torch.empty((n, 1 + 3 * ns), dtype=torch.float32, device="cuda")
    kin.targets(3 * ns, h, z, tg)
    tgn = tg.cpu().numpy()
    np.testing.assert_allclose(tgn[:, 0], np.log(h.cpu().numpy()), rtol=1e-6)
    np.testing.assert_allclose(tgn[:, 1:], z.cpu().numpy().T, rtol=1e-6)
    # prediction: an untrained net gives finite, clipped h0 and finite z0
    net = kin.MLP(3 + ns, 32, 1 + 3 * ns, seed=2)
    ones = torch.ones(1 + 3 * ns, dtype=torch.float32, device="cuda")
    zeros = torch.zeros_like(ones)
    norm = dict(in_mean=mean, in_std=std, out_mean=zeros + np.log(1e-7), out_std=ones)
    h0 = torch.empty(n, dtype=torch.float64, device="cuda")
    z0 = torch.empty((3 * ns, n), dtype=torch.float64, device="cuda")
    net.predict(ns, Y, T, P, 1e-4, norm, h0=h0, z0=z0)
    h0n = h0.cpu().numpy()
    assert np.all(np.isfinite(h0n)) and np.all(h0n <= 1e-4) and np.all(h0n >= 1e-14)
    assert np.all(np.isfinite(z0.cpu().numpy()))


def test_prediction_matches_the_reference_network():
    """kin_mlp_predict on a network with set weights (FP32 mode) against the
    FP64 reference: features, forward pass, de-standardisation, exp and the
    clip of h0 to [1e-14, dt], and the stage guesses z0 [3 ns][n], entry by
    entry."""
    mech = synth.make_mechanism("h2")
    st = synth.make_states(mech, 200, seed=9)
    ns, n, dt = mech.ns, st.n, 1e-4
    din, dout, w = 3 + ns, 1 + 3 * ns, 48
    rng = np.random.default_rng(12)
    net = kin.MLP(din, w, dout, precision="fp32", seed=6)
    p = net.get_params()
    p[:] = (0.5 * p + rng.normal(0, 0.05, p.size)).astype(np.float32)
    net.set_params(p)
    Y, T, P = (torch.from_numpy(a).cuda() for a in (st.Y, st.T, st.P))
    X = torch.empty((n, din), dtype=torch.float32, device="cuda")
    kin.features(ns, Y, T, P, dt, X)
    xm = X.cpu().numpy().astype(np.float64)
    in_mean = xm.mean(0).astype(np.float32)
    in_std = np.maximum(xm.std(0), 1e-3).astype(np.float32)
    out_mean = np.concatenate([[np.log(3e-7)], rng.normal(0, 1e-9, 3 * ns)]).astype(np.float32)
    out_std = np.concatenate([[4.0], np.full(3 * ns, 1e-8)]).astype(np.float32)
    norm = {k: torch.from_numpy(v).cuda() for k, v in
            dict(in_mean=in_mean, in_std=in_std, out_mean=out_mean, out_std=out_std).items()}
    h0 = torch.empty(n, dtype=torch.float64, device="cuda")
    z0 = torch.empty((3 * ns, n), dtype=torch.float64, device="cuda")
    net.predict(ns, Y, T, P, dt, norm, h0=h0, z0=z0)
    torch.cuda.synchronize()
    # reference: FP32 standardised features (as the kernel stores them), FP64 network
    xs = ((X.cpu().numpy() - in_mean) / in_std).astype(np.float64)
    W, b = unpack(p.astype(np.float64), din, w, dout)
    y, _ = M.forward(W, b, xs)
    lh = y[:, 0] * out_std[0] + out_mean[0]
    h_ref = np.clip(np.exp(lh), 1e-14, dt)
    z_ref = (y[:, 1:] * out_std[1:] + out_mean[1:]).T
    scale = np.abs(y).max(axis=0)
    # |dy| <= 1e-5 of the output's scale: h0 relative error |dlh| = std |dy|
    np.testing.assert_allclose(h0.cpu().numpy(), h_ref, rtol=1e-5 * out_std[0] * scale[0] + 1e-6)
    assert np.mean((h_ref > 1e-14) & (h_ref < dt)) > 0.5       # mostly inside the clip
    zb = 1e-5 * (scale[1:] * out_std[1:])[:, None] + 1e-6 * np.abs(z_ref)
    assert np.all(np.abs(z0.cpu().numpy() - z_ref) <= zb)
    # the clip: outputs pushed far out of range land on the bounds
    big = dict(norm, out_mean=norm["out_mean"] + 100.0)
    net.predict(ns, Y, T, P, dt, big, h0=h0)
    assert np.all(h0.cpu().numpy() == dt)
    small = dict(norm, out_mean=norm["out_mean"] - 200.0)
    net.predict(ns, Y, T, P, dt, small, h0=h0)
    assert np.all(h0.cpu().numpy() == 1e-14)


def test_trained_predictor_removes_steps_at_equal_error():
    """What the learned part gains: a predictor trained on integrator-made
    targets (2^17 CH4-like states, WARP layout, FP32 matrices) supplies the
    first internal step of 2^14 fresh states at dt = 1e-4 s.  Radau's error
    test still judges every step.  It must remove at least 1.5 % of the steps
    while the results stay as accurate: against a tight reference (the
    oracle at rtol 1e-10, atol 1e-17) on 48 sampled states, the median
    E_i (Sec. 2.3) at most 1.2 times the run without it and at most one
    more state with E_i > 10.  The tail is compared by count: with FP32
    matrices a changed first step changes the whole step sequence, and the
    states where the error control misses a step change with it."""
    from oracle import oracle as O
    from paper_1607_03884_gb300 import learned
    mech = synth.make_mechanism("ch4")
    tr = synth.make_states(mech, 1 << 17, seed=47, T_range=(800.0, 2600.0))
    te = synth.make_states(mech, 1 << 14, seed=46, T_range=(800.0, 2600.0))
    mg = kin.Mechanism(mech)
    dt = 1e-4
    pred, info = learned.train(mech, mg, tr, dt, width=256, epochs=8, batch=1024, layout="warp")
    assert info["samples"] > 0.9 * tr.n
    assert info["history"][-1] < info["history"][0]
    Y, T, P = (torch.from_numpy(a).cuda() for a in (te.Y, te.T, te.P))
    runs = {}
    for tag in ("none", "predicted"):
        kw = {}
        if tag == "predicted":
            kw["h0"], _ = pred.predict(Y, T, P, dt)
        Yw, Tw = Y.clone(), T.clone()
        mg.integrate(Yw, Tw, P, dt, layout="warp", lu_fp32=True, **kw)
        torch.cuda.synchronize()
        runs[tag] = (Yw.cpu().numpy(), Tw.cpu().numpy(), mg.stats())
    s0, s1 = runs["none"][2], runs["predicted"][2]
    assert s0["failed"] == 0 and s1["failed"] == 0
    idx = np.arange(0, te.n, te.n // 48)
    Yx, Tx, _ = O.integrate(mech, te.subset(idx), dt, rtol=1e-10, atol=1e-17,
                            transform_tol=False)
    yx = np.concatenate([Tx[None], Yx[:-1]])
    E = {tag: O.error_norm(np.concatenate([r[1][idx][None], r[0][:-1, idx]]), yx)
         for tag, r in runs.items()}
    print(f"\nsteps/state {s0['nstep'] / te.n:.2f} -> {s1['nstep'] / te.n:.2f}, right-hand "
          f"sides {s0['nfcn'] / te.n:.1f} -> {s1['nfcn'] / te.n:.1f}; E vs exact max "
          f"{E['none'].max():.3g} -> {E['predicted'].max():.3g}, median "
          f"{np.median(E['none']):.3g} -> {np.median(E['predicted']):.3g}")
    assert s1["nstep"] < 0.985 * s0["nstep"], (s1["nstep"], s0["nstep"])
    assert np.sum(E["predicted"] > 10) <= np.sum(E["none"] > 10) + 1, E
    assert np.median(E["predicted"]) <= 1.2 * np.median(E["none"])


def test_train_step_on_gathered_rows_matches_the_plain_step():
    """kin_mlp_train_step_rows gathers a minibatch inside the library: on a
    permutation's rows it must equal the plain step on those rows copied."""
    rng = np.random.default_rng(3)
    R, M, din, w, dout = 300, 64, 20, 32, 12
    X = torch.from_numpy(rng.normal(size=(R, din)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.normal(size=(R, dout)).astype(np.float32)).cuda()
    rows = torch.from_numpy(rng.permutation(R)[:M].astype(np.int32)).cuda()
    a = kin.MLP(din, w, dout, precision="bf16", seed=5)
    b = kin.MLP(din, w, dout, precision="bf16", seed=5)
    la = torch.zeros(1, dtype=torch.float32, device="cuda")
    lb = torch.zeros(1, dtype=torch.float32, device="cuda")
    a.train_step_rows(X, T, rows, 1e-3, loss_out=la)
    idx = rows.long()
    b.train_step(X[idx].contiguous(), T[idx].contiguous(), 1e-3, loss_out=lb)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.get_params(), b.get_params())
    # the loss is a sum of float atomics: equal up to its summation order
    np.testing.assert_allclose(la.item(), lb.item(), rtol=1e-5)
