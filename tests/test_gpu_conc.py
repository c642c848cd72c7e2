"""GPU parity of the concentration-based form with its sparse LU
(kin_integrate_conc) against the oracle's concentration-based form
(oracle/chem.c orc_rhs_conc, batch form 1) on the same seeded inputs.

Bar, as for the mass-fraction path: with FP64 Newton matrices every
non-igniting state (oracle |dT| <= 10 K) meets 1e-5 in T and in every mass
fraction above 1e-8; T meets it on every state; the igniting states'
error is reported and their accuracy judged against a tight reference
(reading r19).  FP32 matrices are judged by equal accuracy (r19)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_1607_03884_gb300 import kin, synth  # noqa: E402
from test_gpu_parity import (RTOL_PARITY, dev, equal_accuracy, parity,  # noqa: E402
                             split_report)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kin.lib()


def run_conc(cm, st, dt, **opt):
    Y, T, P = dev(st.Y), dev(st.T), dev(st.P)
    n = st.n
    status = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros((8, n), dtype=torch.int32, device="cuda")
    cm.integrate(Y, T, P, dt, status=status, counters=cnt, **opt)
    torch.cuda.synchronize()
    return Y.cpu().numpy(), T.cpu().numpy(), cnt.cpu().numpy().T.copy(), status.cpu().numpy()


@pytest.fixture(scope="module")
def h2c():
    mech, st, _ = synth.workload("h2_1024")
    return mech, kin.ConcMechanism(mech), st


@pytest.fixture(scope="module")
def ch4c():
    mech = synth.make_mechanism("ch4")
    st = synth.make_states(mech, 96, seed=44, T_range=(800.0, 2600.0))
    return mech, kin.ConcMechanism(mech), st


@pytest.mark.parametrize("dt", [1e-6, 1e-4])
def test_h2_conc_parity(h2c, dt):
    mech, cm, st = h2c
    sub = st.subset(np.arange(0, st.n, 2))
    Yo, To, co = O.integrate(mech, sub, dt, form="conc")
    Yg, Tg, cg, sg = run_conc(cm, sub, dt)
    assert np.all(sg == 0) and np.all(co[:, 7] == 0)
    per, relT, quiet, E = split_report(f"H2 conc FP64, dt {dt:g}", Yg, Tg, Yo, To, sub.T)
    assert np.all(per[quiet] <= RTOL_PARITY), np.sort(per[quiet])[-5:]
    assert relT.max() <= RTOL_PARITY
    equal_accuracy(f"H2 conc FP64, dt {dt:g}", mech, sub, dt, Yg, Tg, Yo, To,
                   np.where(per > RTOL_PARITY)[0])
    # the same step sequence on most states (rounding may move a decision)
    assert np.mean(np.all(cg[:, :7] == co[:, :7], axis=1)) >= 0.9


@pytest.mark.parametrize("dt", [1e-6, 1e-4])
def test_ch4_conc_parity(ch4c, dt):
    mech, cm, st = ch4c
    Yo, To, co = O.integrate(mech, st, dt, form="conc")
    Yg, Tg, cg, sg = run_conc(cm, st, dt)
    assert np.all(sg == 0) and np.all(co[:, 7] == 0)
    per, relT, quiet, E = split_report(f"CH4 conc FP64, dt {dt:g}", Yg, Tg, Yo, To, st.T)
    assert np.all(per[quiet] <= RTOL_PARITY), np.sort(per[quiet])[-5:]
    assert relT.max() <= RTOL_PARITY
    equal_accuracy(f"CH4 conc FP64, dt {dt:g}", mech, st, dt, Yg, Tg, Yo, To,
                   np.where(per > RTOL_PARITY)[0])
    assert np.mean(np.all(cg[:, :7] == co[:, :7], axis=1)) >= 0.9


def test_ch4_conc_fp32_matrices(ch4c):
    mech, cm, st = ch4c
    dt = 1e-4
    Yo, To, co = O.integrate(mech, st, dt, form="conc")
    Yg, Tg, cg, sg = run_conc(cm, st, dt, lu_fp32=True)
    assert np.all(sg == 0)
    per, relT, quiet, E = split_report("CH4 conc FP32", Yg, Tg, Yo, To, st.T)
    assert np.median(E) < 1.0
    equal_accuracy("CH4 conc FP32", mech, st, dt, Yg, Tg, Yo, To, np.where(per > RTOL_PARITY)[0])


def test_conc_form_against_the_mass_fraction_form(ch4c):
    """The same reactor in other variables: the GPU's concentration-based
    results are as accurate as the mass-fraction oracle's against a tight
    reference."""
    mech, cm, st = ch4c
    sub = st.subset(np.arange(24))
    dt = 1e-4
    Ym, Tm, cm_ = O.integrate(mech, sub, dt)
    Yg, Tg, cg, sg = run_conc(cm, sub, dt)
    assert np.all(sg == 0)
    equal_accuracy("CH4 conc GPU vs mass-fraction oracle", mech, sub, dt, Yg, Tg, Ym, Tm,
                   np.arange(sub.n))


def test_conc_edge_sizes_ragged_and_empty(h2c):
    mech, cm, st = h2c
    for n in (1, 33):
        sub = st.subset(np.arange(n))
        Yo, To, co = O.integrate(mech, sub, 1e-6, form="conc")
        Yg, Tg, cg, sg = run_conc(cm, sub, 1e-6)
        assert np.all(sg == 0)
        eT, eY, per = parity(Yg, Tg, Yo, To)
        assert eT <= RTOL_PARITY and eY <= RTOL_PARITY, (n, eT, eY)
    Y = torch.zeros((mech.ns, 0), dtype=torch.float64, device="cuda")
    T = torch.zeros(0, dtype=torch.float64, device="cuda")
    cm.integrate(Y, T, T, 1e-6)                       # n = 0 is a no-op
    assert cm.stats()["nstep"] == 0


def test_conc_is_deterministic(ch4c):
    mech, cm, st = ch4c
    sub = st.subset(np.arange(48))
    for opt in (dict(), dict(lu_fp32=True)):
        runs = [run_conc(cm, sub, 1e-6, **opt) for _ in range(3)]
        for r in runs[1:]:
            for a, b in zip(runs[0], r):
                np.testing.assert_array_equal(a, b)


def test_conc_order_and_totals(h2c):
    """A permutation of the states gives the same per-state results (the
    integration of a state does not depend on its slot) and the totals
    match the per-state counters."""
    mech, cm, st = h2c
    sub = st.subset(np.arange(200))
    a = run_conc(cm, sub, 1e-6)
    tot = cm.stats()
    assert tot["nstep"] == int(a[2][:, 0].sum()) and tot["failed"] == 0
    order = torch.from_numpy(np.random.default_rng(1).permutation(sub.n).astype(np.int32)).cuda()
    b = run_conc(cm, sub, 1e-6, order=order)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_conc_rejects_unsupported_options(h2c):
    mech, cm, st = h2c
    sub = st.subset(np.arange(4))
    for opt in (dict(jac_fd=True), dict(layout="plain"), dict(lanes=16), dict(h_fixed=1e-8)):
        with pytest.raises(kin.KinError) as e:
            run_conc(cm, sub, 1e-6, **opt)
        assert e.value.code == kin.KIN_ERR_UNSUPPORTED, opt
