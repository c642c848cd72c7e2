"""Pins of the exprb43 oracle (oracle/exprb.py): the phi functions against
their closed forms and series, the Arnoldi relation, exactness on linear
problems (the scheme reduces to the exact flow when g is constant), the
order conditions of the tableau through the convergence orders on a
nonlinear problem (4 for the solution, 3 for the embedded one), the Krylov
stopping rule (a looser kappa never takes more dimensions), and an
adaptive reactor integration against the tight Radau reference."""
import math

import numpy as np
import pytest

from oracle import exprb as X
from oracle import oracle as O
from paper_1607_03884_gb300 import synth


def phi_series(z, k, terms=40):
    return sum(z ** j / math.factorial(j + k) for j in range(terms))


def phi_closed(z, k):
    """phi_k(z) = (e^z - sum_{j<k} z^j / j!) / z^k for z away from 0."""
    return (math.exp(z) - sum(z ** j / math.factorial(j) for j in range(k))) / z ** k


@pytest.mark.parametrize("z", [-40.0, -3.0, -0.5, 1e-3, 0.7, 2.0])
def test_phi_functions_on_scalars(z):
    ph = X.phi_vectors(np.array([[z]]), 5)
    for k in range(1, 6):
        ref = phi_series(z, k) if abs(z) < 1 else phi_closed(z, k)
        assert abs(ph[k - 1][0] - ref) <= 1e-13 * max(1.0, abs(ref)), (z, k)


def test_phi_functions_of_a_diagonalisable_matrix():
    rng = np.random.default_rng(2)
    lam = np.array([-50.0, -2.0, -0.3, 0.4])
    Q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
    A = Q @ np.diag(lam) @ Q.T
    e1 = np.eye(4)[:, 0]
    ph = X.phi_vectors(A, 3)
    for k in (1, 2, 3):
        ref = Q @ np.diag([phi_closed(z, k) for z in lam]) @ Q.T @ e1
        np.testing.assert_allclose(ph[k - 1], ref, rtol=1e-11, atol=1e-14)


def test_arnoldi_relation_and_exhaustion():
    rng = np.random.default_rng(3)
    N = 9
    J = rng.normal(size=(N, N))
    v = rng.normal(size=N)
    scal = np.ones(N)
    beta, V, H, m = X.arnoldi(J, v, 1e-3, X.PRODUCTS_F, scal, 0.0)   # kappa 0: to the end
    assert m == N
    np.testing.assert_allclose(V.T @ V, np.eye(N), atol=1e-12)
    np.testing.assert_allclose(J @ V, V @ H, atol=1e-11)              # exhausted: exact
    np.testing.assert_allclose(beta * V[:, 0], v, rtol=1e-14)
    # with error weights the space is that of D^-1 J D from D^-1 v
    sc = rng.uniform(0.1, 10.0, size=N)
    beta, V, H, m = X.arnoldi(J, v, 1e-3, X.PRODUCTS_F, sc, 0.0)
    Js = J * sc[None, :] / sc[:, None]
    np.testing.assert_allclose(V.T @ V, np.eye(N), atol=1e-12)
    np.testing.assert_allclose(Js @ V, V @ H, atol=1e-10)
    np.testing.assert_allclose(beta * V[:, 0] * sc, v, rtol=1e-13)
    # a looser kappa never takes more dimensions
    ms = [X.arnoldi(J, v, 1e-3, X.PRODUCTS_F, scal, k)[3] for k in (0.0, 1e-12, 1e-6, 1e-2, 1.0)]
    assert all(a >= b for a, b in zip(ms, ms[1:])) and ms[-1] < N


def test_linear_problems_are_integrated_exactly():
    """y' = A y + b: g = b is constant, D2 = D3 = 0 and one step is the exact
    flow e^{hA} y + h phi1(hA) b (exact Krylov space, weighted)."""
    rng = np.random.default_rng(4)
    N = 6
    Q, _ = np.linalg.qr(rng.normal(size=(N, N)))
    A = Q @ np.diag(-np.logspace(-1, 4, N)) @ Q.T
    b = rng.normal(size=N)
    y0 = rng.normal(size=N)
    f = lambda v: A @ v + b
    y, st = X.integrate(f, lambda v: A, y0, 0.1, kappa=0.0, hfixed=0.1)
    assert st["naccpt"] == 1
    exact = expm_flow(A, b, y0, 0.1)
    np.testing.assert_allclose(y, exact, rtol=1e-11, atol=1e-12)


def expm_flow(A, b, y0, t):
    from scipy.linalg import expm
    N = len(y0)
    M = np.zeros((N + 1, N + 1))
    M[:N, :N] = A * t
    M[:N, N] = b * t
    return (expm(M) @ np.concatenate([y0, [1.0]]))[:N]


def _nonlinear():
    """A mildly stiff nonlinear 3-species system with a smooth solution."""
    def f(y):
        return np.array([-20.0 * y[0] + y[1] * y[2],
                         y[0] - 2.0 * y[1] ** 2 + 0.5 * y[2],
                         -y[2] + 0.3 * y[0] * y[1]])

    def J(y):
        return np.array([[-20.0, y[2], y[1]],
                         [1.0, -4.0 * y[1], 0.5],
                         [0.3 * y[1], 0.3 * y[0], -1.0]])
    return f, J, np.array([1.0, 0.5, 2.0])


def test_convergence_orders_four_and_three():
    """Constant steps, exact Krylov spaces: the solution's global error falls
    16x per halving (order 4: the order conditions sum b_i c_i^2/2 = phi3
    and sum b_i c_i^3/6 = phi4 hold), the embedded solution's 8x (order 3)."""
    from scipy.integrate import solve_ivp
    f, J, y0 = _nonlinear()
    t1 = 1.0
    ref = solve_ivp(lambda t, y: f(y), (0, t1), y0, method="Radau", rtol=1e-13, atol=1e-15,
                    jac=lambda t, y: J(y)).y[:, -1]
    errs, errs_hat = [], []
    for n in (40, 80, 160):
        h = t1 / n
        y = y0.copy()
        yh = y0.copy()
        for _ in range(n):
            fy = f(y)
            unew, _, _, _ = X.step(f, J(y), y, fy, h, np.ones(3), 0.0)
            fyh = f(yh)
            _, uhat, _, _ = X.step(f, J(yh), yh, fyh, h, np.ones(3), 0.0)
            y, yh = unew, uhat
        errs.append(np.abs(y - ref).max())
        errs_hat.append(np.abs(yh - ref).max())
    r = [errs[i] / errs[i + 1] for i in range(2)]
    rh = [errs_hat[i] / errs_hat[i + 1] for i in range(2)]
    assert all(14.0 < q < 18.0 for q in r), (errs, r)
    assert all(7.0 < q < 9.0 for q in rh), (errs_hat, rh)


def test_adaptive_reactor_integration_meets_the_tolerance():
    """H2 states over dt = 1e-6 s at rtol 1e-6, atol 1e-10: E_i against the
    tight Radau reference of order one or below, as the paper reports for
    its exponential solvers (Sec. 2.3)."""
    mech, st, _ = synth.workload("h2_1024")
    sub = st.subset(np.arange(0, 1024, 128))
    Y, T, stats = X.integrate_states(mech, sub, 1e-6)
    assert all(s["status"] == 0 for s in stats)
    Yx, Tx, cx = O.integrate(mech, sub, 1e-6, rtol=1e-13, atol=1e-20, transform_tol=False)
    E = O.error_norm(np.concatenate([T[None], Y[:-1]]), np.concatenate([Tx[None], Yx[:-1]]))
    assert np.median(E) < 1.0 and E.max() < 20.0, E
    assert max(s["krylov_max"] for s in stats) <= mech.ns
