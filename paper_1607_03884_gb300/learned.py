"""Training and use of the step/guess predictor (host orchestration only).

Every computation runs in libkin: the integrator produces the training
trajectories (first accepted step and its converged stages), the kin_mlp_*
kernels build features and targets, standardise them, train the network
and predict; this module only sequences those calls.

Targets.  For each training state the first internal step the integrator
would accept when it starts as large as possible is found by starting it at
h0 = dt and letting the error test shrink it (pass 1, a few step attempts
only); pass 2 starts again from that step and records the converged stage
increments of the first step.  The network learns (log h0, Z0) from
(log T, log P, log dt, log10 Y).  At use time Radau keeps its error test and
step control: a prediction that is too large is rejected and shrunk like any
first step.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import kin


@dataclasses.dataclass
class Predictor:
    net: "kin.MLP"
    norm: dict          # device float tensors in_mean, in_std, out_mean, out_std
    ns: int

    def scaled(self, factor):
        """The same network with its first-step prediction multiplied by
        factor (a shift of the ln h0 output's mean; no extra kernel)."""
        norm = {k: v.clone() for k, v in self.norm.items()}
        norm["out_mean"][0:1] += float(np.log(factor))
        return Predictor(net=self.net, norm=norm, ns=self.ns)

    def predict(self, Y, T, P, dt, stream=None):
        import torch
        n = int(T.shape[0])
        h0 = torch.empty(n, dtype=torch.float64, device=T.device)
        z0 = torch.empty((3 * self.ns, n), dtype=torch.float64, device=T.device)
        self.net.predict(self.ns, Y, T, P, dt, self.norm, h0=h0, z0=z0, stream=stream)
        return h0, z0


def first_step_targets(mg, states, dt, rtol=1e-6, atol=1e-10, max_attempts=60, lu_fp32=True,
                       chunk=1 << 18, layout="plain"):
    """(mask, h, z) on the device: the largest-accepted first step and its
    converged stages for each state (mask: the state produced both)."""
    import torch
    n, N = states.n, mg.ns
    hs, zs, ok = [], [], []
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        sub = states.subset(np.arange(a, b))
        m = b - a
        Y = torch.from_numpy(sub.Y).cuda()
        T = torch.from_numpy(sub.T).cuda()
        P = torch.from_numpy(sub.P).cuda()
        h_try = torch.full((m,), float(dt), dtype=torch.float64, device="cuda")
        h1 = torch.zeros(m, dtype=torch.float64, device="cuda")
        mg.integrate(Y.clone(), T.clone(), P, dt, rtol, atol, h0=h_try, h_first=h1,
                     max_steps=max_attempts, stop_after=1, lu_fp32=lu_fp32, layout=layout)
        good = h1 > 0
        h_use = torch.where(good, h1, h_try)
        h2 = torch.zeros(m, dtype=torch.float64, device="cuda")
        z2 = torch.zeros((3 * N, m), dtype=torch.float64, device="cuda")
        mg.integrate(Y.clone(), T.clone(), P, dt, rtol, atol, h0=h_use, h_first=h2, z_first=z2,
                     max_steps=max_attempts, stop_after=1, lu_fp32=lu_fp32, layout=layout)
        good = good & (h2 > 0)
        hs.append(h2)
        zs.append(z2)
        ok.append(good)
    return torch.cat(ok), torch.cat(hs), torch.cat(zs, dim=1)


def train(mech, mg, states, dt, *, width=256, epochs=4, batch=4096, lr=2e-3, seed=0,
          precision="bf16", rtol=1e-6, atol=1e-10, layout="plain", h_weight=None, log=None):
    """Generate targets with the integrator and train a predictor on them.

    The loss is the mean squared error of the standardised outputs; the
    first-step output is given the weight of all stage outputs together
    (h_weight, default 3N) by shrinking its standardisation scale, since it
    is the output that changes the integration most.
    """
    import torch
    ns = mech.ns
    din, dout = 3 + ns, 1 + 3 * ns
    mask, h, z = first_step_targets(mg, states, dt, rtol, atol, layout=layout)
    idx = torch.nonzero(mask).flatten()
    Y = torch.from_numpy(states.Y).cuda()[:, idx].contiguous()
    T = torch.from_numpy(states.T).cuda()[idx].contiguous()
    P = torch.from_numpy(states.P).cuda()[idx].contiguous()
    h = h[idx].contiguous()
    z = z[:, idx].contiguous()
    n = int(idx.numel())
    X = torch.empty((n, din), dtype=torch.float32, device="cuda")
    kin.features(ns, Y, T, P, dt, X)
    Tg = torch.empty((n, dout), dtype=torch.float32, device="cuda")
    kin.targets(3 * ns, h, z, Tg)
    norm = {k: torch.empty(d, dtype=torch.float32, device="cuda")
            for k, d in (("in_mean", din), ("in_std", din), ("out_mean", dout), ("out_std", dout))}
    kin.moments(X, norm["in_mean"], norm["in_std"])
    kin.moments(Tg, norm["out_mean"], norm["out_std"])
    w = float(h_weight if h_weight is not None else 3 * ns)
    norm["out_std"][0:1] /= w ** 0.5
    Xs = torch.empty_like(X)
    kin.features(ns, Y, T, P, dt, Xs, norm["in_mean"], norm["in_std"])
    Ts = torch.empty_like(Tg)
    kin.targets(3 * ns, h, z, Ts, norm["out_mean"], norm["out_std"])
    net = kin.MLP(din, width, dout, precision=precision, seed=seed)
    rng = np.random.default_rng(seed)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    history = []
    steps = max(1, n // batch)
    for ep in range(epochs):
        # a host-drawn permutation per epoch; the library gathers each batch
        perm = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
        lr_ep = lr * (0.5 ** ep)
        acc = 0.0
        for s in range(steps):
            net.train_step_rows(Xs, Ts, perm[s * batch:(s + 1) * batch], lr_ep, loss_out=loss)
            acc += loss.item() if (s % 16 == 0) else 0.0
        history.append(acc / max(1, (steps + 15) // 16))
        if log:
            log(f"epoch {ep}: mean loss {history[-1]:.4f}")
    return Predictor(net=net, norm=norm, ns=ns), dict(samples=n, history=history)
