"""Pins of the oracle's Radau IIA core against closed forms and exact solutions.

The oracle derives its tableau, transformation and error weights numerically
from the collocation nodes; these tests hold it to the textbook closed forms
(tests/golden), to the method's stability function (the (2,3) Pade
approximant of exp), to its classical order 5, and to the exact solution of
a stiff linear system (the matrix exponential).
"""
import numpy as np
import pytest
import scipy.linalg

from conftest import load_closed_forms
from oracle import oracle as O


@pytest.fixture(scope="module")
def tb():
    return O.tableau()


def test_tableau_matches_closed_forms(tb):
    g = load_closed_forms()
    np.testing.assert_allclose(tb["c"], [g["c1"], g["c2"], g["c3"]], rtol=0, atol=1e-15)
    A = np.array([[g["a11"], g["a12"], g["a13"]], [g["a21"], g["a22"], g["a23"]],
                  [g["a31"], g["a32"], g["a33"]]])
    np.testing.assert_allclose(tb["A"], A, rtol=0, atol=2e-15)
    np.testing.assert_allclose(tb["b"], A[2], rtol=0, atol=2e-15)
    np.testing.assert_allclose(tb["e"] / tb["gamma0"], [g["d1"], g["d2"], g["d3"]], rtol=1e-13)


def test_tableau_order_conditions(tb):
    A, b, c = tb["A"], tb["b"], tb["c"]
    for k in range(1, 6):          # B(5): quadrature order 5 (order 2s-1)
        assert abs(b @ c ** (k - 1) - 1.0 / k) < 1e-14
    for k in range(1, 4):          # C(3): stage order 3
        np.testing.assert_allclose(A @ c ** (k - 1), c ** k / k, atol=1e-15)


def test_transformation_block_diagonalises_Ainv(tb):
    Ai = np.linalg.inv(tb["A"])
    ev = np.linalg.eigvals(Ai)
    real = ev[np.abs(ev.imag) < 1e-12].real
    cplx = ev[ev.imag > 1e-12]
    assert abs(real[0] - tb["gamma"]) < 1e-12
    assert abs(cplx[0].real - tb["alpha"]) < 1e-12
    assert abs(cplx[0].imag - tb["beta"]) < 1e-12
    L = tb["TI"] @ Ai @ tb["T"]
    want = np.array([[tb["gamma"], 0, 0], [0, tb["alpha"], -tb["beta"]],
                     [0, tb["beta"], tb["alpha"]]])
    np.testing.assert_allclose(L, want, atol=1e-13)
    np.testing.assert_allclose(tb["TI"] @ tb["T"], np.eye(3), atol=1e-14)
    # normalisation: unit real eigenvector with positive last entry, complex
    # eigenvector with last entry exactly 1 (T[2,1] = 1, T[2,2] = 0)
    assert abs(np.linalg.norm(tb["T"][:, 0]) - 1.0) < 1e-15 and tb["T"][2, 0] > 0
    assert abs(tb["T"][2, 1] - 1.0) < 1e-15 and abs(tb["T"][2, 2]) < 1e-15
    assert abs(tb["gamma0"] * tb["gamma"] - 1.0) < 1e-15


def _R(z):
    g = load_closed_forms()
    num = sum(c * z ** k for k, c in enumerate(g["R_num"]))
    den = sum(c * z ** k for k, c in enumerate(g["R_den"]))
    return num / den


@pytest.mark.parametrize("lam", [-0.5, -5.0, -50.0, -1e4, -1e8, 0.3])
def test_one_step_is_stability_function_real(lam):
    h = 0.1
    y, st = O.radau(lambda t, y: lam * y, lambda t, y: np.array([[lam]]), [1.0], 0.0, h,
                    hfixed=h, rtol=1e-12, atol=1e-20)
    assert st["nstep"] == 1 and st["status"] == 0
    assert abs(y[0] - _R(h * lam)) <= 1e-13 * max(1.0, abs(_R(h * lam)))


@pytest.mark.parametrize("a,b", [(-1.0, 3.0), (-20.0, 100.0), (-0.1, 2.0), (-1e5, 1e3)])
def test_one_step_is_stability_function_complex(a, b):
    """y' = [[a,-b],[b,a]] y has eigenvalue a+ib; one step maps x+iy by R(h(a+ib))."""
    M = np.array([[a, -b], [b, a]])
    h = 0.05
    y0 = np.array([0.7, -0.2])
    y, st = O.radau(lambda t, y: M @ y, lambda t, y: M, y0, 0.0, h, hfixed=h, rtol=1e-12,
                    atol=1e-20)
    w = _R(h * complex(a, b)) * complex(y0[0], y0[1])
    assert st["status"] == 0
    np.testing.assert_allclose(y, [w.real, w.imag], rtol=0, atol=1e-13 * max(1, abs(w)))


def test_classical_order_five_on_smooth_problem():
    """Logistic y' = y (1 - y): constant steps, global error ~ h^5 (ratio 32)."""
    y0, t1 = 0.1, 2.0
    exact = 1.0 / (1.0 + (1.0 / y0 - 1.0) * np.exp(-t1))
    errs = []
    for m in (10, 20, 40):
        y, st = O.radau(lambda t, y: y * (1 - y), lambda t, y: np.array([[1 - 2 * y[0]]]),
                        [y0], 0.0, t1, hfixed=t1 / m, rtol=1e-13, atol=1e-20)
        assert st["status"] == 0 and st["naccpt"] == m
        errs.append(abs(y[0] - exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 26 < r1 < 40 and 26 < r2 < 40, errs


def _stiff_linear(n=5, seed=3):
    rng = np.random.default_rng(seed)
    lam = -np.logspace(0, 8, n)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    V = Q @ np.diag(rng.uniform(0.5, 2.0, n))
    A = V @ np.diag(lam) @ np.linalg.inv(V)
    y0 = rng.uniform(0.5, 1.5, n)
    return A, y0, V, lam


@pytest.mark.parametrize("t1", [1e-6, 1e-3, 1.0])
def test_adaptive_on_stiff_linear_system_matches_matrix_exponential(t1):
    A, y0, V, lam = _stiff_linear()
    exact = V @ np.diag(np.exp(lam * t1)) @ np.linalg.solve(V, y0)
    np.testing.assert_allclose(exact, scipy.linalg.expm(A * t1) @ y0, rtol=1e-8, atol=1e-12)
    y, st = O.radau(lambda t, y: A @ y, lambda t, y: A, y0, 0.0, t1, rtol=1e-6, atol=1e-10)
    assert st["status"] == 0
    E = np.sqrt(np.mean(((y - exact) / (1e-10 + 1e-6 * np.abs(exact))) ** 2))
    assert E < 10.0, (E, st)
    # a tighter tolerance gets closer: the controller responds to rtol
    y2, st2 = O.radau(lambda t, y: A @ y, lambda t, y: A, y0, 0.0, t1, rtol=1e-10, atol=1e-14)
    assert np.max(np.abs(y2 - exact)) < np.max(np.abs(y - exact)) + 1e-15
    assert st2["naccpt"] >= st["naccpt"]


def test_jacobian_reuse_on_linear_problem():
    """On a linear problem Newton contracts at once, so after an accepted step
    the reuse rule keeps J; only a rejected step taken with a stale J asks for
    a fresh one.  So every Jacobian beyond the first follows a rejection."""
    A, y0, _, _ = _stiff_linear()
    y, st = O.radau(lambda t, y: A @ y, lambda t, y: A, y0, 0.0, 1.0, rtol=1e-6, atol=1e-10)
    rejected = st["nstep"] - st["naccpt"]
    assert 1 <= st["njac"] <= 1 + rejected
    assert st["ndec"] <= st["nstep"]
    assert st["naccpt"] > 3 * st["njac"]


def test_initial_stage_guess_is_used_and_reported():
    """A first-step stage guess equal to the converged stages needs one Newton
    iteration; the reported first-step stages are those converged stages."""
    lam = -3.0
    n = 1
    zf = np.zeros(3 * n)
    y, st = O.radau(lambda t, y: lam * y, lambda t, y: np.array([[lam]]), [1.0], 0.0, 0.1,
                    hfixed=0.1, rtol=1e-10, atol=1e-14, z_first_out=zf)
    y2, st2 = O.radau(lambda t, y: lam * y, lambda t, y: np.array([[lam]]), [1.0], 0.0, 0.1,
                      hfixed=0.1, rtol=1e-10, atol=1e-14, z0=zf.copy())
    assert st2["nsol"] < st["nsol"]
    np.testing.assert_allclose(y2, y, rtol=1e-12)
    # stage values of the collocation solution of y' = lam y: Z = (I - h lam A)^-1 h lam A 1
    tb = O.tableau()
    Z = np.linalg.solve(np.eye(3) - 0.1 * lam * tb["A"], 0.1 * lam * tb["A"] @ np.ones(3))
    np.testing.assert_allclose(zf, Z, rtol=1e-10)


def test_max_steps_status_keeps_last_accepted_state():
    A, y0, _, _ = _stiff_linear()
    y, st = O.radau(lambda t, y: A @ y, lambda t, y: A, y0, 0.0, 1.0, rtol=1e-6, atol=1e-10,
                    max_steps=3)
    assert st["status"] == 1 and st["naccpt"] <= 3
    assert np.all(np.isfinite(y))


def test_final_step_below_round_off_of_t_ends_the_integration():
    """Reading of the fixed global step (Sec. 2.3): a last step shorter than
    the round-off of t means the state is already at t1, so the integration
    ends there (status 0, the state unchanged) instead of reporting a step
    size underflow.  A step that short anywhere else is still an underflow."""
    lam = -1.0
    y, st = O.radau(lambda t, v: lam * v, lambda t, v: np.array([[lam]]), [1.0],
                    1.0, 1.0 + 4e-16)
    assert st["status"] == 0 and st["nstep"] == 1 and st["naccpt"] == 0
    assert y[0] == 1.0
    # a remainder of a few ulps of t still takes an ordinary step
    y, st = O.radau(lambda t, v: lam * v, lambda t, v: np.array([[lam]]), [1.0],
                    1.0, 1.0 + 1e-13)
    assert st["status"] == 0 and st["naccpt"] == 1
    np.testing.assert_allclose(y[0], np.exp(lam * 1e-13), rtol=1e-15)
    # a step forced below round-off before the end is an underflow
    y, st = O.radau(lambda t, v: lam * v, lambda t, v: np.array([[lam]]), [1.0],
                    1.0, 2.0, h0=1e-18)
    assert st["status"] == 2


def test_error_estimate_scales_as_h_to_the_fourth():
    """The embedded estimate (order-3 companion of the order-5 method) is a
    local error of order h^4 on a smooth problem: its ratio per halving of a
    constant step tends to 2^4.  Measured on the second of two steps, so the
    first-step refinement does not enter."""
    lam = -1.0
    hs = [0.1, 0.05, 0.025, 0.0125]
    errs = []
    for h in hs:
        y, st = O.radau(lambda t, v: lam * v, lambda t, v: np.array([[lam]]), [1.0], 0.0,
                        2 * h, hfixed=h, rtol=1e-10, atol=1e-10, transform_tol=False)
        assert st["status"] == 0 and st["naccpt"] == 2
        errs.append(st["err_last"])
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.diff(ratios) > 0), ratios          # approaching the asymptote
    assert 15.0 <= ratios[-1] <= 17.0, ratios


@pytest.mark.parametrize("kind,idx,dt", [("h2", (0, 256, 512, 768), 1e-6), ("ch4", (1,), 1e-7)])
def test_tight_solution_agrees_with_scipy_radau(kind, idx, dt):
    """The oracle at rtol 1e-13 (the 'exact' reference of the error studies)
    against scipy's independent Radau IIA at rtol 1e-12 on the same right-hand
    side and Jacobian: T and every species above 1e-8 agree to 1e-11."""
    from scipy.integrate import solve_ivp
    from paper_1607_03884_gb300 import synth
    mech = synth.make_mechanism(kind)
    if kind == "h2":
        _, st, _ = synth.workload("h2_1024")
    else:
        st = synth.make_states(mech, 8, seed=44, T_range=(800.0, 2600.0))
    st = st.subset(np.array(idx))
    om = O.OracleMech(mech)
    y0 = O.state_vector(st)
    Yx, Tx, _ = O.integrate(mech, st, dt, rtol=1e-13, atol=1e-20, transform_tol=False)
    yx = np.concatenate([Tx[None], Yx[:-1]])
    for i in range(st.n):
        P = st.P[i]
        r = solve_ivp(lambda t, v: O.rhs(om, P, v)[0], (0.0, dt), y0[:, i], method="Radau",
                      jac=lambda t, v: O.jac(om, P, v)[0], rtol=1e-12, atol=1e-20)
        assert r.status == 0
        big = np.abs(yx[:, i]) > 1e-8
        rel = np.abs(r.y[big, -1] - yx[big, i]) / np.abs(yx[big, i])
        assert rel.max() < 1e-11, (i, rel.max())
