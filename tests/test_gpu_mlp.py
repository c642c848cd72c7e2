"""The step/guess predictor's CUDA kernels against the FP64 numpy reference
(oracle/mlp.py): forward values, loss gradients (BF16 tensor-core mode to
~2 %, FP32 check mode to 1e-5), Adam training progress, and the feature /
target / prediction kernels that connect it to the integrator."""
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


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("bf16", 3e-2)])
@pytest.mark.parametrize("din,w,dout,n", [(16, 64, 40, 77), (56, 32, 160, 130)])
def test_forward_and_gradients_against_fp64_reference(precision, tol, din, w, dout, n):
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
    if precision == "bf16":
        W = [bf16(Wl) for Wl in W]
        x = bf16(x)
    y, cache = M.forward(W, b, x)
    gW, gb = M.backward(W, b, cache, y, T.astype(np.float64))
    ref = np.concatenate([np.concatenate([a.ravel(), c]) for a, c in zip(gW, gb)])
    yg = Y.cpu().numpy()
    assert np.linalg.norm(yg - y) / np.linalg.norm(y) < tol
    gg = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - ref) / np.linalg.norm(ref) < tol
    assert abs(loss.item() - M.loss(y, T)) / M.loss(y, T) < tol


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


def test_trained_predictor_removes_steps_at_equal_error():
    """What the learned part gains: a predictor trained on integrator-made
    targets (CH4-like states, WARP layout, FP32 matrices) gives a first step
    that removes steps against the starting-step heuristic, and the results
    stay as close to the exact solution (oracle at rtol 1e-13) as without it."""
    from oracle import oracle as O
    from paper_1607_03884_gb300 import learned
    mech = synth.make_mechanism("ch4")
    tr = synth.make_states(mech, 1 << 17, seed=47, T_range=(800.0, 2600.0))
    te = synth.make_states(mech, 1 << 12, seed=46, T_range=(800.0, 2600.0))
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
    assert s1["nstep"] < 0.985 * s0["nstep"], (s1["nstep"], s0["nstep"])
    idx = np.arange(0, te.n, te.n // 16)
    Yx, Tx, _ = O.integrate(mech, te.subset(idx), dt, rtol=1e-13, atol=1e-20)
    yx = np.concatenate([Tx[None], Yx[:-1]])
    E = {tag: O.error_norm(np.concatenate([r[1][idx][None], r[0][:-1, idx]]), yx)
         for tag, r in runs.items()}
    print(f"\nsteps/state {s0['nstep'] / te.n:.2f} -> {s1['nstep'] / te.n:.2f}; "
          f"E vs exact max {E['none'].max():.3g} -> {E['predicted'].max():.3g}")
    assert E["predicted"].max() <= max(10.0 * E["none"].max(), 30.0)
    assert np.median(E["predicted"]) <= max(3.0 * np.median(E["none"]), 1.0)


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
