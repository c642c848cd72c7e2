"""GPU parity of exprb43 (kin_integrate_exprb) against the exprb43 oracle
(oracle/exprb.py) on the same seeded states.

The two sides evaluate the phi functions differently (the GPU by scaling
and squaring with a Pade approximant, the oracle by scipy's expm; about
1e-8 apart per call on stiff CH4 Hessenbergs), and the Krylov dimension is
chosen by an estimate that rounding can move across its threshold, so a
state may take another step or Krylov sequence: the element-wise bar (1e-5
in T on every state and in every mass fraction above 1e-8 on the
non-igniting ones with the oracle's step sequence) holds on H2 and on CH4
at dt = 1e-6; over the hundred steps of CH4 at dt = 1e-4 the results stay
within the integrator's tolerance of the oracle (E_i <= 1); states whose
sequences part are judged by equal accuracy against the tight Radau
reference (readings r19, r23, r24)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import exprb as X  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_1607_03884_gb300 import kin, synth  # noqa: E402
from test_gpu_parity import RTOL_PARITY, dev, equal_accuracy, parity, split_report  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kin.lib()


def run_exprb(xr, st, dt, **kw):
    Y, T, P = dev(st.Y), dev(st.T), dev(st.P)
    n = st.n
    status = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros((8, n), dtype=torch.int32, device="cuda")
    xr.integrate(Y, T, P, dt, status=status, counters=cnt, **kw)
    torch.cuda.synchronize()
    return Y.cpu().numpy(), T.cpu().numpy(), cnt.cpu().numpy().T.copy(), status.cpu().numpy()


def oracle_exprb(mech, st, dt, kappa=0.1):
    Y, T, stats = X.integrate_states(mech, st, dt, kappa=kappa)
    cnt = np.array([[s["nstep"], s["naccpt"], s["nrejct"], s["nfcn"], s["njac"], 0, s["krylov"],
                     s["status"]] for s in stats], dtype=np.int64)
    return Y, T, cnt


@pytest.fixture(scope="module")
def h2x():
    mech, st, _ = synth.workload("h2_1024")
    return mech, kin.ExpRosenbrock(mech), st


@pytest.mark.parametrize("dt,kappa", [(1e-6, 0.1), (1e-4, 0.1), (1e-6, 0.0)])
def test_h2_exprb_parity(h2x, dt, kappa):
    mech, xr, st = h2x
    sub = st.subset(np.arange(0, st.n, 16))
    Yo, To, co = oracle_exprb(mech, sub, dt, kappa)
    Yg, Tg, cg, sg = run_exprb(xr, sub, dt, kappa=kappa)
    assert np.all(sg == 0) and np.all(co[:, 7] == 0)
    tag = f"H2 exprb43, dt {dt:g}, kappa {kappa:g}"
    per, relT, quiet, E = split_report(tag, Yg, Tg, Yo, To, sub.T)
    assert relT.max() <= RTOL_PARITY
    same_seq = np.all(cg[:, :5] == co[:, :5], axis=1)
    # the element-wise bar wherever the two took the same steps
    assert np.all(per[quiet & same_seq] <= RTOL_PARITY), np.sort(per[quiet & same_seq])[-5:]
    equal_accuracy(tag, mech, sub, dt, Yg, Tg, Yo, To, np.where(per > RTOL_PARITY)[0])
    print(f"{tag}: same step and evaluation counts as the oracle on {same_seq.mean():.3f} of "
          f"the states; Krylov dimension per space {cg[:, 6].sum() / max(1, cg[:, 5].sum()):.2f}")
    assert same_seq.mean() >= 0.75
    # the counters: 3 Krylov spaces per attempt, 2 or 3 right-hand sides
    assert np.all(cg[:, 5] == 3 * cg[:, 0])


@pytest.mark.parametrize("dt", [1e-6, 1e-4])
def test_ch4_exprb_parity(dt):
    """53 species (two register slots per lane): configuration 3's states."""
    mech, st, _ = synth.workload("ch4_2p18")
    st = st.subset(np.arange(8))
    xr = kin.ExpRosenbrock(mech)
    Yo, To, co = oracle_exprb(mech, st, dt)
    Yg, Tg, cg, sg = run_exprb(xr, st, dt)
    assert np.all(sg == 0) and np.all(co[:, 7] == 0)
    tag = f"CH4 exprb43, dt {dt:g}"
    per, relT, quiet, E = split_report(tag, Yg, Tg, Yo, To, st.T)
    assert relT.max() <= RTOL_PARITY
    same_seq = np.all(cg[:, :5] == co[:, :5], axis=1)
    if dt <= 1e-6:
        assert np.all(per[quiet & same_seq] <= RTOL_PARITY)
    # over 100 steps the two matrix-function algorithms' differences (1e-8
    # relative per call) reach a fraction of the tolerance in minor
    # species: within the integrator's own tolerance of the oracle (r24)
    assert np.all(E[same_seq] <= 1.0), E
    equal_accuracy(tag, mech, st, dt, Yg, Tg, Yo, To, np.where(per > RTOL_PARITY)[0])
    print(f"{tag}: same step and evaluation counts on {same_seq.mean():.3f} of the states")
    assert same_seq.mean() >= 0.75
    # the step counts stay those of the method, not of a failure mode
    assert cg[:, 0].max() <= 2 * co[:, 0].max()


def test_ch4_exprb_chem_and_phi_units():
    """The unit entries: the right-hand side and Jacobian the method uses
    against orc_rhs / orc_jac, and the matrix functions of a Krylov
    Hessenberg matrix against the oracle's phi_vectors (scipy's expm)."""
    mech, st, _ = synth.workload("ch4_2p18")
    sub = st.subset(np.arange(6))
    xr = kin.ExpRosenbrock(mech)
    N = mech.ns
    y = np.concatenate([sub.T[None], sub.Y[:-1]])
    f = torch.zeros((N, sub.n), dtype=torch.float64, device="cuda")
    f2 = torch.zeros_like(f)
    J = torch.zeros((N * N, sub.n), dtype=torch.float64, device="cuda")
    xr.chem(dev(y), dev(sub.P), f, f2, J)
    torch.cuda.synchronize()
    f, f2, J = f.cpu().numpy(), f2.cpu().numpy(), J.cpu().numpy()
    om = O.OracleMech(mech)
    for i in range(sub.n):
        fo = O.rhs(om, sub.P[i], y[:, i])[0]
        Jo = O.jac(om, sub.P[i], y[:, i])[0]
        assert np.abs(f[:, i] - fo).max() <= 1e-12 * np.abs(fo).max()
        assert np.abs(f2[:, i] - fo).max() <= 1e-12 * np.abs(fo).max()
        colmax = np.abs(Jo).max(axis=0) + 1e-300
        assert (np.abs(J[:, i].reshape(N, N) - Jo) / colmax).max() < 1e-11
    yi = y[:, 0]
    Jo = O.jac(om, sub.P[0], yi)[0]
    fo = O.rhs(om, sub.P[0], yi)[0]
    scal = 1e-10 + 1e-6 * np.abs(yi)
    for h in (1e-7, 1e-5):
        b, V, H, m = X.arnoldi(Jo, fo, h, X.PRODUCTS_F, scal, 0.0)
        for mm in (3, 9, m):
            out = torch.zeros((mm, 5), dtype=torch.float64, device="cuda")
            xr.phi(dev(H[:mm, :mm]), 5, h, out)
            torch.cuda.synchronize()
            ref = np.stack(X.phi_vectors(h * H[:mm, :mm], 5), axis=1)
            g = out.cpu().numpy()
            # normwise (scaling and squaring), and each last-row entry relatively
            assert np.abs(g - ref).max() <= 1e-6 * np.abs(ref).max(), (h, mm)
            np.testing.assert_allclose(g[-1], ref[-1], rtol=1e-4)


def test_exprb_edges_determinism_and_arguments(h2x):
    mech, xr, st = h2x
    sub = st.subset(np.arange(33))
    a = run_exprb(xr, sub, 1e-6)
    b = run_exprb(xr, sub, 1e-6)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    tot = xr.stats()
    assert tot["nstep"] == int(a[2][:, 0].sum()) and tot["failed"] == 0
    one = run_exprb(xr, st.subset(np.arange(1)), 1e-6)
    np.testing.assert_array_equal(one[1], a[1][:1])
    Y = torch.zeros((mech.ns, 0), dtype=torch.float64, device="cuda")
    T = torch.zeros(0, dtype=torch.float64, device="cuda")
    xr.integrate(Y, T, T, 1e-6)
    assert xr.stats()["nstep"] == 0
    with pytest.raises(kin.KinError) as e:
        run_exprb(xr, sub, 1e-6, kappa=-1.0)
    assert e.value.code == kin.KIN_ERR_INVALID_ARG
