"""kin_integrate_static: the entry point for callers that cannot allocate
device memory (their host framework's allocator owns it, or they must not
allocate once running).  It takes the mechanism as a host description and
works in libkin's fixed device array instead of a kin_mech's cudaMalloc'd
workspace.  It runs the one-state-per-thread kernel with FP64 matrices, so
its results must equal, bit for bit, kin_integrate_ex's with that layout on
the same inputs, call after call (the array keeps the previous call's
contents, so the second call checks that everything that must start at zero
is cleared), and a call must not change the device's free memory.  This
file is collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1607_03884_gb300 import kin, synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kin.lib()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _reference(mech, st, dt):
    """kin_integrate_ex with the static entry's configuration."""
    mg = kin.Mechanism(mech)
    Y, T, P = _dev(st.Y), _dev(st.T), _dev(st.P)
    s = torch.zeros(st.n, dtype=torch.int32, device="cuda")
    mg.integrate(Y, T, P, dt, status=s, layout="plain", block=64)
    torch.cuda.synchronize()
    return Y.cpu().numpy(), T.cpu().numpy(), s.cpu().numpy()


def _static(mech, st, dt):
    Y, T, P = _dev(st.Y), _dev(st.T), _dev(st.P)
    s = torch.full((st.n,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    kin.integrate_static(mech, Y, T, P, dt, status=s)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    return Y.cpu().numpy(), T.cpu().numpy(), s.cpu().numpy(), free0, free1


@pytest.mark.parametrize("kind,n,dt", [("h2", 777, 1e-5), ("ch4", 96, 1e-6)])
def test_static_entry_matches_workspace_entry(kind, n, dt):
    mech = synth.make_mechanism(kind)
    st = synth.make_states(mech, n, seed=31, T_range=(900.0, 2500.0))
    Yr, Tr, sr = _reference(mech, st, dt)
    for call in range(2):                             # two calls in a row
        Ys, Ts, ss, free0, free1 = _static(mech, st, dt)
        np.testing.assert_array_equal(Ts, Tr)
        np.testing.assert_array_equal(Ys, Yr)
        np.testing.assert_array_equal(ss, sr)
        if call == 1:                                 # set-up done: nothing allocated
            assert free1 == free0, (free0, free1)


def _repeat_reactions(mech, nr):
    """The mechanism with its reactions repeated cyclically up to nr reactions
    (duplicate reactions are a valid mechanism: their rates add)."""
    big = synth.Mechanism(**{**mech.__dict__})
    idx = np.arange(nr) % mech.nr
    big.nr = nr
    for f in ("reac", "prod", "arrh", "eff", "fall", "rtype"):
        setattr(big, f, np.ascontiguousarray(getattr(mech, f)[idx]))
    return big


def test_static_entry_at_its_size_limit():
    """The largest mechanism whose tables fit the 64 KiB array (found by
    bisection over repeated CH4 reactions, with empty batches that only
    upload tables) integrates to the same bits as the workspace entry, and
    one more reaction is rejected."""
    mech = synth.make_mechanism("ch4")
    empty = synth.make_states(mech, 4, seed=1).subset(np.arange(0))

    def fits(nr):
        try:
            kin.integrate_static(_repeat_reactions(mech, nr), _dev(empty.Y), _dev(empty.T),
                                 _dev(empty.P), 1e-6)
            return True
        except kin.KinError as e:
            assert e.code == kin.KIN_ERR_UNSUPPORTED
            return False

    lo, hi = mech.nr, 8 * mech.nr                      # lo fits, hi does not
    assert fits(lo) and not fits(hi)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        lo, hi = (mid, hi) if fits(mid) else (lo, mid)
    big = _repeat_reactions(mech, lo)
    print(f"\nlargest static mechanism: {big.ns} species, {big.nr} reactions")
    st = synth.make_states(mech, 40, seed=3, T_range=(900.0, 2500.0))
    Yr, Tr, sr = _reference(big, st, 1e-7)
    Ys, Ts, ss, _, _ = _static(big, st, 1e-7)
    np.testing.assert_array_equal(Ts, Tr)
    np.testing.assert_array_equal(Ys, Yr)
    np.testing.assert_array_equal(ss, sr)
    with pytest.raises(kin.KinError) as e:
        kin.integrate_static(_repeat_reactions(mech, lo + 1), _dev(st.Y), _dev(st.T),
                             _dev(st.P), 1e-7)
    assert e.value.code == kin.KIN_ERR_UNSUPPORTED


def test_static_entry_refuses_stream_capture():
    """A graph captured from the static entry would replay table uploads from
    host memory the call has freed, so it refuses a capturing stream."""
    mech = synth.make_mechanism("h2")
    st = synth.make_states(mech, 8, seed=2)
    Y, T, P = _dev(st.Y), _dev(st.T), _dev(st.P)
    kin.integrate_static(mech, Y, T, P, 1e-6)          # set-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        with pytest.raises(kin.KinError) as e:
            kin.integrate_static(mech, Y, T, P, 1e-6)
    assert e.value.code == kin.KIN_ERR_UNSUPPORTED
