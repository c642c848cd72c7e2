"""kin_integrate_static: the entry point for callers that cannot allocate
device memory (their host framework's allocator owns it, or they must not
allocate once running).  It takes the mechanism as a host description and
works in libkin's fixed device array instead of a kin_mech's cudaMalloc'd
workspace.  Its results must equal kin_integrate_ex's with default options
on the same inputs, call after call (the array keeps the previous call's
contents, so the second call checks that everything that must start at zero
is cleared).  This file is collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1607_03884_gb300 import kin, synth  # noqa: E402

pytestmark = pytest.mark.gpu

RTOL_PARITY = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kin.lib()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    mask = np.abs(b) > 1e-8
    return float(np.max(np.where(mask, np.abs(a - b) / np.where(mask, np.abs(b), 1.0), 0.0)))


@pytest.mark.parametrize("kind,n,dt", [("h2", 777, 1e-5), ("ch4", 96, 1e-6)])
def test_static_entry_matches_workspace_entry(kind, n, dt):
    mech = synth.make_mechanism(kind)
    st = synth.make_states(mech, n, seed=31, T_range=(900.0, 2500.0))
    mg = kin.Mechanism(mech)
    Yr, Tr, P = _dev(st.Y), _dev(st.T), _dev(st.P)
    sr = torch.zeros(n, dtype=torch.int32, device="cuda")
    mg.integrate(Yr, Tr, P, dt, status=sr)            # kin_integrate_ex, default options
    torch.cuda.synchronize()
    for call in range(2):                             # two calls in a row
        Ys, Ts = _dev(st.Y), _dev(st.T)
        ss = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        kin.integrate_static(mech, Ys, Ts, P, dt, status=ss)
        torch.cuda.synchronize()
        assert _rel(Ts.cpu().numpy(), Tr.cpu().numpy()) <= RTOL_PARITY, call
        assert _rel(Ys.cpu().numpy(), Yr.cpu().numpy()) <= RTOL_PARITY, call
        np.testing.assert_array_equal(ss.cpu().numpy(), sr.cpu().numpy())


def test_static_entry_rejects_tables_beyond_its_array():
    mech = synth.make_mechanism("ch4")
    big = synth.Mechanism(**{**mech.__dict__})
    reps = 8                                          # 8 x 325 reactions: > 64 KiB of tables
    big.nr = mech.nr * reps
    for f in ("reac", "prod", "arrh", "eff", "fall"):
        setattr(big, f, np.concatenate([getattr(mech, f)] * reps))
    big.rtype = np.concatenate([mech.rtype] * reps)
    st = synth.make_states(mech, 4, seed=1)
    with pytest.raises(kin.KinError) as e:
        kin.integrate_static(big, _dev(st.Y), _dev(st.T), _dev(st.P), 1e-6)
    assert e.value.code == kin.KIN_ERR_UNSUPPORTED
