"""Benchmark: integrated reactor states per second for one global step.

Workload: the seeded H2/O2-like mechanism (13 species, 27 reactions) on 2^20
PaSR-like states (20 % near-equilibrium products, 80 % ignition-delay
states, random order), one global step dt (default 1e-4 s; 1e-6 s is also
reported), rtol 1e-6, atol 1e-10.  The launch configuration is autotuned
(kin_autotune on a 2^18-state prefix).  A timed step is one replay of a CUDA
graph holding the stiffness ordering (kin_order_states) and one integration
of the whole batch; inputs are restored from a pristine device copy and L2
is flushed (256 MiB write) before every timed step, outside the timed
region.  After the timed steps it measures, untimed for the headline: the
plain FP64 one-state-per-thread kernel on the same states and the error
between the two, the other dt, the warp divergence D, the same integration
through the host-buffer entry (copies included), and the oracle on a
sample of the states on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --workload ch4_2p18 --layout warp ...   (other workloads)

Under torchrun each rank integrates its own copy of the workload (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "h2_mixed_2p20"
METRIC = "integrated states/sec per global step (dt=1e-6, 1e-4 s) vs plain FP64 GPU Radau, equal error"
RTOL, ATOL = 1e-6, 1e-10


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--dt", type=float, default=1e-4)
    p.add_argument("--workload", default=WORKLOAD,
                   help="a named synthetic workload (synth.WORKLOADS); the metric's is the default")
    p.add_argument("--layout", default="auto", choices=["auto", "plain", "queue", "warp"])
    p.add_argument("--lanes", type=int, default=0, choices=[0, 4, 8, 16, 32],
                   help="lanes per state for --layout warp (0 = 32)")
    p.add_argument("--jac", default="analytic", choices=["analytic", "fd"],
                   help="analytical or finite-difference Jacobian")
    p.add_argument("--fp32", type=int, default=1, help="FP32 Newton matrices (1) or FP64 (0)")
    p.add_argument("--n", type=int, default=0, help="states (0 = the workload's 2^20)")
    p.add_argument("--no-extras", action="store_true", help="skip the comparison legs")
    p.add_argument("--no-config3", action="store_true",
                   help="skip the full-size CH4-like and predictor legs among the extras")
    p.add_argument("--config5", action="store_true",
                   help="only the learned part at full size (2^20 training and test states)")
    p.add_argument("--config3-only", default=None, choices=["massfrac", "conc"],
                   help="time only configuration 3 in the given form (states = --n, default "
                        "2^18)")
    p.add_argument("--exprb-only", action="store_true",
                   help="time only exprb43 on the first --n states (default 2^16) at --dt")
    p.add_argument("--mlp-only", action="store_true",
                   help="time only the predictor's training step (rows = --n, default 2^16)")
    p.add_argument("--cpu-sample", type=int, default=2048)
    p.add_argument("--order", default="heuristic", choices=["none", "heuristic"],
                   help="order the states by the starting-step heuristic inside each step")
    p.add_argument("--graph", type=int, default=1,
                   help="replay the integration as a captured CUDA graph (1) or call it (0)")
    return p.parse_args()


# ---------------------------------------------------------------------------
# algorithmic operation counts (FP64 / FP32 flops per event)
# ---------------------------------------------------------------------------

def op_model(mech, form="massfrac"):
    """Counted operations per event for this mechanism (oracle/flop_counts.json,
    written by oracle/opcount.py; transcendentals count as one operation), or
    None when the mechanism has no committed count.  form "conc": the
    concentration-based form with its sparse LU."""
    from oracle import opcount
    rec = opcount.load_counts(mech, form)
    return None if rec is None else opcount.per_event(rec)


def algorithmic_flops(tot, ops, fp32):
    """(FP64, FP32) operations of one launch from its summed counters.

    Events: right-hand sides (nfcn), Jacobians beyond their point's f (njac),
    factorisation pairs (ndec), Newton iterations (nsol: both solves and the
    iteration's algebra), error estimates (at least naccpt + nrejct: every
    accepted step and every error-test rejection after the first acceptance;
    the uncounted ones make this a lower bound), step attempts (nstep) and
    accepted steps (naccpt).  With FP32 Newton matrices the factorisations,
    the solves and the Jacobian assembly are FP32 work."""
    nerr = tot["naccpt"] + tot["nrejct"]
    lin = tot["ndec"] * ops["lu_linear"] + tot["nsol"] * ops["sol_linear"] + nerr * ops["err_linear"]
    jac = tot["njac"] * ops["jac"]
    total = (tot["nfcn"] * ops["rhs"] + jac + tot["ndec"] * ops["lu"] + tot["nsol"] * ops["sol"]
             + nerr * ops["err"] + tot["nstep"] * ops["step"] + tot["naccpt"] * ops["accept"])
    if not fp32:
        return float(total), 0.0
    f32 = lin + jac
    return float(total - f32), float(f32)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------

def max_over_ranks(t, dist=None, device="cpu"):
    """The slowest rank's step time (every rank gets it); t itself on one rank."""
    if dist is None:
        return float(t)
    import torch
    tt = torch.tensor([float(t)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(n_per_rank, world, t_max):
    """States per second of the whole job: every rank integrates its own n
    states (weak scaling, no collective on the data path), the job lasts as
    long as its slowest rank."""
    return n_per_rank * world / t_max


def run_ours(args, rank, world):
    import torch
    from paper_1607_03884_gb300 import kin, synth

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    mech, st, _ = synth.workload(args.workload, n=args.n or None)
    n = st.n
    mg = kin.Mechanism(mech)
    Y0 = torch.from_numpy(st.Y).cuda()
    T0 = torch.from_numpy(st.T).cuda()
    P = torch.from_numpy(st.P).cuda()
    Y, T = Y0.clone(), T0.clone()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    ops = op_model(mech)
    tune = None
    if args.layout == "auto":
        # autotuner (kin_autotune) on a 2^18-state prefix: layout, block, refill batch
        m = min(n, 1 << 18)
        best, secs = mg.autotune(Y0[:, :m].contiguous(), T0[:m].contiguous(), P[:m].contiguous(),
                                 args.dt, RTOL, ATOL, stream=stream, lu_fp32=bool(args.fp32),
                                 jac_fd=args.jac == "fd")
        tune = {"states": m, "best": best, "candidate_seconds": [round(x, 4) for x in secs],
                "candidates": "plain 64/32, queue 64 refill 1/4/8/16/32, queue 32, "
                              "warp lanes 32/16/8/4 (-1: skipped)"}
        opt = dict(layout=best["layout"], block=best["block"], queue_refill=best["queue_refill"],
                   lanes=best["lanes"], lu_fp32=bool(args.fp32), jac_fd=args.jac == "fd")
    else:
        opt = dict(layout=args.layout, lu_fp32=bool(args.fp32), jac_fd=args.jac == "fd",
                   lanes=args.lanes)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    graph = None
    if args.graph:
        # one memset node + one integration kernel node, replayed each step
        graph = mg.capture(Y, T, P, args.dt, RTOL, ATOL,
                           order_by=None if args.order == "none" else args.order, **opt)
    ordered = args.order != "none"
    key_buf = torch.empty(n, dtype=torch.float64, device="cuda")
    order_buf = torch.empty(n, dtype=torch.int32, device="cuda")

    def one(dt, o, timed, g=None, ordered=False):
        Y.copy_(Y0)
        T.copy_(T0)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if g is not None:
            g.replay()
        elif ordered:
            mg.order_states(Y, T, P, RTOL, ATOL, key=key_buf, order=order_buf, stream=stream)
            mg.integrate(Y, T, P, dt, RTOL, ATOL, stream=stream, order=order_buf, **o)
        else:
            mg.integrate(Y, T, P, dt, RTOL, ATOL, stream=stream, **o)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3

    for _ in range(args.warmup):
        one(args.dt, opt, False, graph, ordered)
    barrier()
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    wall0 = time.perf_counter()
    times = [one(args.dt, opt, True, graph, ordered) for _ in range(args.steps)]
    barrier()
    wall = time.perf_counter() - wall0
    clocks = clk.stop()
    tot = mg.stats()
    t_step = float(np.mean(times))
    t_median = float(np.median(times))
    t_max = max_over_ranks(t_step, dist, "cuda")
    value = whole_job_rate(n, world, t_max)
    f64, f32 = algorithmic_flops(tot, ops, bool(args.fp32)) if ops else (None, None)

    out = {"tune": tune, "opt": {k: v for k, v in opt.items()}}
    if rank == 0 and not args.no_extras:
        Y_ours, T_ours = Y.cpu().numpy(), T.cpu().numpy()
        # the plain FP64 one-state-per-thread kernel on the same workload
        base_opt = dict(layout="plain", lu_fp32=False)
        one(args.dt, base_opt, False)
        tb = [one(args.dt, base_opt, True) for _ in range(max(1, min(args.steps, 2)))]
        out["plain_fp64_states_per_s"] = n / float(np.mean(tb))
        # equal error: the paper's E_i (Sec. 2.3) of our result against the
        # plain FP64 kernel's, at the requested tolerances
        yo = np.concatenate([T_ours[None], Y_ours[:-1]])
        yb = np.concatenate([T.cpu().numpy()[None], Y.cpu().numpy()[:-1]])
        E = np.sqrt(np.mean(((yo - yb) / (ATOL + np.abs(yb) * RTOL)) ** 2, axis=0))
        out["error_vs_plain_fp64"] = {"E_max": float(E.max()), "E_median": float(np.median(E)),
                                      "E_p99": float(np.percentile(E, 99))}
        # dt = 1e-6 for both
        other = 1e-6 if args.dt != 1e-6 else 1e-4
        one(other, opt, False, None, ordered)
        t_o = float(np.mean([one(other, opt, True, None, ordered) for _ in range(2)]))
        one(other, base_opt, False)
        t_ob = float(np.mean([one(other, base_opt, True) for _ in range(2)]))
        out["per_dt"] = {str(args.dt): {"ours": value / world, "plain_fp64": out["plain_fp64_states_per_s"]},
                         str(other): {"ours": n / t_o, "plain_fp64": n / t_ob}}
        # end to end through the host-buffer entry (pinned buffers)
        Yh = torch.from_numpy(st.Y.copy()).pin_memory()
        Th = torch.from_numpy(st.T.copy()).pin_memory()
        Ph = torch.from_numpy(st.P.copy()).pin_memory()
        Yp = Yh.clone().pin_memory()
        Tp = Th.clone().pin_memory()
        hopt = dict(opt, order_by=None if args.order == "none" else args.order)
        mg.integrate_host(Yp, Tp, Ph, args.dt, RTOL, ATOL, stream=stream, **hopt)
        te = []
        for _ in range(max(1, min(args.steps, 3))):
            Yp.copy_(Yh)
            Tp.copy_(Th)
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mg.integrate_host(Yp, Tp, Ph, args.dt, RTOL, ATOL, stream=stream, **hopt)
            te.append(time.perf_counter() - t0)
        # warp divergence D = 1 - sum d / (32 max d) per warp of 32 consecutive
        # slots (Sec. 3.3), from the per-state step counts d; a state's steps do
        # not depend on its slot, so one counted run gives D for any order
        Y.copy_(Y0)
        T.copy_(T0)
        cnt = torch.zeros((8, n), dtype=torch.int32, device="cuda")
        mg.integrate(Y, T, P, args.dt, RTOL, ATOL, stream=stream, counters=cnt,
                     **{k: v for k, v in opt.items() if k != "order"})
        mg.order_states(Y0, T0, P, RTOL, ATOL, key=key_buf, order=order_buf, stream=stream)
        torch.cuda.synchronize()
        d = cnt[0].cpu().numpy().astype(np.float64)

        def warp_div(v):
            w = v[: v.size // 32 * 32].reshape(-1, 32)
            return float(np.mean(1.0 - w.sum(1) / (32.0 * np.maximum(w.max(1), 1.0))))
        out["divergence"] = {"D_mean_in_input_order": warp_div(d),
                             "D_mean_ordered": warp_div(d[order_buf.cpu().numpy()]),
                             "steps_mean": float(d.mean()), "steps_max": int(d.max())}
        out["e2e"] = {"value": n / float(np.mean(te)), "unit": "states/s",
                      "h2d_bytes_per_step": int(n * (mech.ns + 2) * 8),
                      "d2h_bytes_per_step": int(n * (mech.ns + 1) * 8)}
    if rank == 0 and not args.no_extras and not args.no_config3 and args.workload == WORKLOAD:
        out["configs"] = {"ch4_2p18": config3_leg(stream),
                          "ch4_2p18_conc": config3_leg(stream, form="conc"),
                          "h2_exprb43": exprb_leg(stream),
                          "mlp_train": mlp_leg(stream)}
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return dict(value=value, t_step=t_max, t_median=t_median, times=times, wall=wall,
                clocks=clocks, tot=tot,
                f64=f64, f32=f32, n=n, mech=mech, st=st, extras=out)


def config3_leg(stream, form="massfrac", n=0):
    """The CH4-like configuration at full size, outside the headline's timed
    region: 2^18 states (53 species, 325 reactions), dt = 1e-4 s, the state-
    per-warp layout with FP32 Newton matrices.  One warm-up launch on a 4096-
    state prefix, then one timed launch of the whole batch (CUDA events on the
    launching stream, L2 flushed before), with its own counted roofline.
    form "conc": the same states in the concentration-based form with its
    sparse LU (kin_integrate_conc; Sec. 3.3, Sec. 4).  n > 0: the first n
    states only."""
    import torch
    from paper_1607_03884_gb300 import kin, synth
    mech, st, _ = synth.workload("ch4_2p18")
    if 0 < n < st.n:
        st = st.subset(np.arange(n))
    conc = form == "conc"
    mg = kin.ConcMechanism(mech) if conc else kin.Mechanism(mech)
    opt = dict(layout="warp", lanes=32, lu_fp32=True)
    Y, T, P = (torch.from_numpy(a.copy()).cuda() for a in (st.Y, st.T, st.P))
    m = min(4096, st.n)
    mg.integrate(Y[:, :m].contiguous(), T[:m].clone(), P[:m].contiguous(), 1e-4, RTOL, ATOL,
                 stream=stream, **opt)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    flush.zero_()
    torch.cuda.synchronize()
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    mg.integrate(Y, T, P, 1e-4, RTOL, ATOL, stream=stream, **opt)
    e1.record(stream)
    e1.synchronize()
    clocks = clk.stop()
    sec = e0.elapsed_time(e1) / 1e3
    tot = mg.stats()
    ops = op_model(mech, form)
    f64, f32 = algorithmic_flops(tot, ops, True) if ops else (None, None)
    kernel = "k_integrate_conc<32, float>" if conc else "k_integrate_lanes<32, float>"
    rec = {"workload": "ch4_2p18", "states": st.n, "species": mech.ns, "reactions": mech.nr,
           "dt": 1e-4, "layout": "warp", "lanes": 32, "newton_matrices": "fp32",
           "form": "concentration-based, sparse LU" if conc else "mass fractions, dense LU",
           "value": st.n / sec, "unit": "states/s", "seconds": sec, "failed": tot["failed"],
           "counters": {k: int(v) for k, v in tot.items()}, "clocks": clocks,
           "roofline": roofline(f64, f32, sec, None, kernel)}
    if conc:
        rec["tolerances"] = "atol on T and V, atol / W_k on the moles n_k (the mass-fraction weights)"
    return rec


def exprb_leg(stream, n=1 << 16, dt=1e-4, kappa=0.1):
    """exprb43 with Krylov phi-function products (kin_integrate_exprb; the
    paper's comparison method, Sec. 2.1, Sec. 3.1) on the first n states of
    the headline workload, outside the headline's timed region: one warm-up
    launch on 256 states, one timed launch (CUDA events, L2 flushed
    before).  Its matrix-function work depends on per-call scaling counts
    the counters do not record, so the leg reports no roofline."""
    import torch
    from paper_1607_03884_gb300 import kin, synth
    mech, st, _ = synth.workload(WORKLOAD)
    st = st.subset(np.arange(n))
    xr = kin.ExpRosenbrock(mech)
    Y, T, P = (torch.from_numpy(a.copy()).cuda() for a in (st.Y, st.T, st.P))
    m = 256
    xr.integrate(Y[:, :m].contiguous(), T[:m].clone(), P[:m].contiguous(), dt, RTOL, ATOL,
                 kappa=kappa, stream=stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    flush.zero_()
    torch.cuda.synchronize()
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    xr.integrate(Y, T, P, dt, RTOL, ATOL, kappa=kappa, stream=stream)
    e1.record(stream)
    e1.synchronize()
    clocks = clk.stop()
    sec = e0.elapsed_time(e1) / 1e3
    tot = xr.stats()
    return {"workload": f"{WORKLOAD} (first {n} states)", "states": n, "dt": dt,
            "method": "exprb43, Krylov tolerance kappa = %g, one state per warp, FP64" % kappa,
            "value": n / sec, "unit": "states/s", "seconds": sec, "failed": tot["failed"],
            "steps_per_state": tot["nstep"] / n,
            "krylov_dim_per_space": tot["krylov_dim"] / max(1, tot["krylov_spaces"]),
            "counters": {k: int(v) for k, v in tot.items()}, "clocks": clocks,
            "roofline": None}


def mlp_leg(stream, rows=1 << 16, steps=20):
    """The predictor's training step on the tensor cores (the learned part's
    GEMMs: 56 -> 256 -> 256 -> 256 -> 160, BF16 operands, FP32 accumulators
    in tensor memory): CUDA-event time of `steps` Adam steps on batches of
    `rows` seeded rows, outside the headline's timed region.  One step runs
    the forward pass (4 GEMMs), the backward pass (4 weight-gradient and 3
    input-gradient GEMMs) and the elementwise kernels."""
    import torch
    from paper_1607_03884_gb300 import kin
    din, w, dout = 56, 256, 160
    net = kin.MLP(din, w, dout, precision="bf16", seed=5)
    g = torch.Generator(device="cpu").manual_seed(11)
    X = torch.randn((rows, din), generator=g).cuda()
    T = torch.randn((rows, dout), generator=g).cuda()
    for _ in range(3):
        net.train_step(X, T, 1e-4, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        net.train_step(X, T, 1e-4, stream=stream)
    e1.record(stream)
    e1.synchronize()
    sec = e0.elapsed_time(e1) / 1e3 / steps
    pad = lambda d, m: (d + m - 1) // m * m
    k0, n3 = pad(din, 16), pad(dout, 8)
    macs = rows * (k0 * w + 2 * w * w + w * n3)            # forward
    flops = 2.0 * macs * 3 - 2.0 * rows * k0 * w          # + weight and input gradients
    pk = peaks().get("bf16_tflops")
    tf = flops / sec / 1e12
    return {"rows": rows, "layers": [din, w, w, w, dout], "seconds_per_step": sec,
            "gemm_tflops": tf, "peak_bf16_tflops": pk, "frac": (tf / pk) if pk else None,
            "note": "GEMM flops of a step over the whole step's time (elementwise kernels "
                    "and Adam included)"}


def config5_leg(stream, n_train=1 << 20, n_test=1 << 20):
    """The learned part at full size: a predictor trained on n_train states
    of `ch4_learned_train_2p20` (targets from the integrator itself), then
    n_test fresh states of `ch4_learned_test_2p20` integrated over dt = 1e-4 s
    (WARP, FP32 Newton matrices) with the starting-step heuristic and with the
    predicted first step: states/s (CUDA events, prediction included) and
    events per state.  Accuracy against the exact solution is a test's job
    (tests/test_gpu_mlp.py)."""
    import torch
    from paper_1607_03884_gb300 import kin, learned, synth
    mech, tr, _ = synth.workload("ch4_learned_train_2p20", n=n_train)
    _, te, _ = synth.workload("ch4_learned_test_2p20", n=n_test)
    mg = kin.Mechanism(mech)
    dt = 1e-4
    t0 = time.perf_counter()
    pred, info = learned.train(mech, mg, tr, dt, width=256, epochs=6, batch=4096, layout="warp")
    train_s = time.perf_counter() - t0
    Y0, T0, P = (torch.from_numpy(a.copy()).cuda() for a in (te.Y, te.T, te.P))
    out = {"train_states": n_train, "test_states": n_test, "train_seconds": train_s,
           "final_loss": info["history"][-1]}
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    for tag in ("heuristic", "predicted"):
        Y, T = Y0.clone(), T0.clone()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        kw = {}
        if tag == "predicted":
            kw["h0"], _ = pred.predict(Y, T, P, dt, stream=stream)
        mg.integrate(Y, T, P, dt, RTOL, ATOL, stream=stream, layout="warp", lu_fp32=True, **kw)
        e1.record(stream)
        e1.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        st = mg.stats()
        out[tag] = {"states_per_s": n_test / sec, "seconds": sec,
                    **{f"{k}_per_state": st[k] / n_test for k in
                       ("nstep", "nfcn", "nsol", "ndec", "njac")}, "failed": st["failed"]}
    out["clocks"] = clk.stop()
    out["step_reduction"] = 1.0 - out["predicted"]["nstep_per_state"] / out["heuristic"]["nstep_per_state"]
    out["speedup"] = out["predicted"]["states_per_s"] / out["heuristic"]["states_per_s"]
    return out


def cpu_model():
    """The host CPU's name as the OS reports it (x86 'model name' or Arm 'CPU part')."""
    try:
        with open("/proc/cpuinfo") as fh:
            txt = fh.read()
    except OSError:
        return None
    for key in ("model name", "CPU part"):
        for line in txt.splitlines():
            if line.startswith(key):
                return f"{key}: {line.split(':', 1)[1].strip()}"
    return None


def cpu_baseline(sample, dt, workload=WORKLOAD, one_core=True):
    from oracle import oracle as O
    from paper_1607_03884_gb300 import synth
    mech, st, _ = synth.workload(workload)
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(st.n, size=sample, replace=False))
    sub = st.subset(idx)
    t0 = time.perf_counter()
    O.integrate(mech, sub, dt, rtol=RTOL, atol=ATOL)
    el = time.perf_counter() - t0
    out = {"value": sample / el, "unit": "states/s", "cores": O.num_threads(), "kind": "oracle",
           "sample": f"{sample} states drawn (seed 1) from the {workload} workload, dt={dt:g}",
           "seconds": el, "cpu": cpu_model(),
           "build": "gcc " + " ".join(O.CFLAGS) + " (the checker's build: IEEE order, no "
                    "FMA contraction, no host-specific instructions; OpenMP over states, "
                    "dynamic schedule of 16)"}
    if one_core:  # the same oracle on one thread, over a quarter of the sample
        m = max(16, sample // 4)
        t0 = time.perf_counter()
        O.integrate(mech, sub.subset(np.arange(m)), dt, rtol=RTOL, atol=ATOL, nthreads=1)
        out["value_1core"] = m / (time.perf_counter() - t0)
    return out


# the sources the thread-per-state kernel is compiled and launched from; the
# state-per-warp header, the ordering, static-entry and predictor sources
# generate none of its code
PLAIN_KERNEL_SOURCES = ("kin_api.cu", "kin_device.cuh", "kin_internal.h", "kin_kernels.cuh",
                        "kin_radau.cuh", "kin_tu_16f.cu")


def kernel_digest():
    """Digest of the sources that define and launch the thread-per-state
    integration kernel, whose DRAM traffic profiles/dram_traffic.json
    records: a traffic figure taken from other sources is void."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1607_03884_gb300", "csrc")
    for name in PLAIN_KERNEL_SOURCES:
        h.update(name.encode())
        with open(os.path.join(d, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def dram_traffic(key, n):
    """DRAM bytes (read + write) of one integration launch over n states, from
    the ncu capture summarised in profiles/dram_traffic.json (bytes per state,
    scaled by states), or None when that capture is of other kernel sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    e = rec.get("kernels", {}).get(key)
    if not e or rec.get("sources_digest") != kernel_digest():
        return None
    return float(e["bytes_per_state"]) * n


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except Exception:
        return {}


# FP64 FMA peak: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz (max SM clock);
# the unit count was measured on this GB300, and a dependent-FMA kernel on all
# SMs reached FP64_PROBE_TFLOPS.  FP32: 152 x 128 lanes x 2 x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP64_PROBE_TFLOPS = 1.198
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def roofline(f64, f32, seconds, traffic=None, kernel=None):
    """The FP64-pipe roofline of one launch from its counted operations."""
    if f64 is None:
        return {"bound": "alu", "achieved": None, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": None, "traffic": traffic, "note": "no committed operation count"}
    a64 = f64 / seconds / 1e12
    return {"bound": "alu", "achieved": a64, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": a64 / FP64_PEAK_TFLOPS, "traffic": traffic, "pipe": "fp64", "kernel": kernel,
            "peak_source": "152 SMs x 2 FP64 FMA/clk x 2.07 GHz (unit count measured)",
            "frac_of_probe_peak": a64 / FP64_PROBE_TFLOPS, "probe_peak": FP64_PROBE_TFLOPS,
            "fp32_tflops": f32 / seconds / 1e12,
            "time_bound_frac": a64 / FP64_PEAK_TFLOPS + f32 / seconds / 1e12 / FP32_PEAK_TFLOPS,
            "flops_source": "operations per event counted by oracle/opcount.py "
                            "(oracle/flop_counts.json) times the launch's event counters",
            "traffic_source": None if traffic is None else
                              "ncu dram__bytes_read+write of a 131072-state capture "
                              "(profiles/dram_traffic.json), scaled by states"}


def main():
    args = parse()
    if args.config5:    # the learned part at full size (minutes; not part of the default run)
        import torch
        print(json.dumps(config5_leg(torch.cuda.current_stream())))
        return
    if args.config3_only:   # configuration 3 alone, in one form (for profiling its kernel)
        import torch
        print(json.dumps(config3_leg(torch.cuda.current_stream(), args.config3_only, args.n)))
        return
    if args.exprb_only:   # exprb43 alone (for profiling its kernel)
        import torch
        print(json.dumps(exprb_leg(torch.cuda.current_stream(), n=args.n or (1 << 16),
                                   dt=args.dt)))
        return
    if args.mlp_only:   # the predictor's training step alone (for profiling its GEMMs)
        import torch
        print(json.dumps(mlp_leg(torch.cuda.current_stream(), rows=args.n or (1 << 16),
                                 steps=args.steps)))
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank != 0:
            return
        reps = []
        for _ in range(args.warmup + args.steps):
            reps.append(cpu_baseline(max(64, args.cpu_sample // 4), args.dt, args.workload,
                                     one_core=False))
        vals = [r["value"] for r in reps[args.warmup:]]
        v = float(np.mean(vals))
        cb = dict(reps[-1])
        cb["value"] = v
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": "states/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * cb["seconds"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "dt": args.dt, "rtol": RTOL, "atol": ATOL,
                       "sample": cb["sample"]},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "states/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}))
        return
    r = run_ours(args, rank, world)
    if rank != 0:
        return
    t = r["t_step"]
    roof = roofline(r["f64"], r["f32"], t,
                    dram_traffic(f"{r['extras']['opt'].get('layout')}:"
                                 f"{'f32' if args.fp32 else 'f64'}", r["n"]),
                    f"k_integrate_{r['extras']['opt'].get('layout')}")
    cb = cpu_baseline(args.cpu_sample, args.dt, args.workload) if not args.no_extras else None
    ex = r["extras"]
    line = {
        "metric": METRIC, "value": r["value"], "unit": "states/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32" if args.fp32 else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "states": r["n"], "species": r["mech"].ns,
                   "reactions": r["mech"].nr, "dt": args.dt, "rtol": RTOL, "atol": ATOL,
                   "layout": ex["opt"].get("layout"), "block": ex["opt"].get("block", 0),
                   "queue_refill": ex["opt"].get("queue_refill", 0),
                   "lanes": ex["opt"].get("lanes", 0), "autotune": ex.get("tune"),
                   "newton_matrices": "fp32" if args.fp32 else "fp64", "jacobian": args.jac,
                   "order": args.order,
                   "l2": "flushed (256 MiB write) and inputs restored before each timed step"},
        "roofline": roof,
        "cpu_baseline": cb,
        "e2e": ex.get("e2e"),
        "ms_per_step_median": 1e3 * r["t_median"],
        # per step: the integration kernel, plus the six ordering kernels
        # (init, key, min/max, histogram, scan, scatter) when ordering
        "gpu_launches": args.steps * (1 + (6 if args.order != "none" else 0)),
        "graph": bool(args.graph),
        "clocks": r["clocks"],
        "plain_fp64_states_per_s": ex.get("plain_fp64_states_per_s"),
        "vs_plain_fp64": (r["value"] / world / ex["plain_fp64_states_per_s"]
                          if ex.get("plain_fp64_states_per_s") else None),
        "error_vs_plain_fp64": ex.get("error_vs_plain_fp64"),
        "per_dt": ex.get("per_dt"),
        "divergence": ex.get("divergence"),
        "configs": ex.get("configs"),
        "counters": {k: int(v) for k, v in r["tot"].items()},
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
