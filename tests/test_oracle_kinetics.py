"""Pins of the oracle's chemistry (thermo, rates, Jacobians) and of what its
integrations must conserve.

What pins what:
* NASA-7 thermo: dh/dT = cp and ds/dT = cp/T (thermodynamic identities),
  and the choice of coefficient set on either side of T_mid.
* Rates: the isothermal A <-> B closed form Y_A(t) = Y_eq + (Y_A0 - Y_eq)
  exp(-(kf + kr) t) (mass action, reverse rate from K_c, the ODE's scaling),
  the Troe factor at log Pr + c = 0 (F = Fcent) and its two limits.
* Jacobians: analytical against a fourth-order central difference of the
  right-hand side (best agreement over a sweep of increments), and the
  CVODE-style one-sided Jacobian against the analytical one.
* Integrations: element conservation (a linear invariant every RK method
  keeps), mixture enthalpy at constant pressure (adiabatic reactor), the
  second law (mixture entropy never decreases), and detailed balance at
  long-time equilibrium against K_c computed here from Gibbs energies.
"""
import copy

import numpy as np
import pytest

from oracle import oracle as O
from paper_1607_03884_gb300 import synth

RU = 8314.46261815324
PATM = 101325.0


# ----------------------------------------------------------------------------
# helpers written here from first principles (not the oracle's code)
# ----------------------------------------------------------------------------

def nasa_eval(nasa_row, T):
    """cp/R, h/RT, s/R of one species from its NASA-7 row (test-side copy)."""
    a = nasa_row[3:10] if T < nasa_row[1] else nasa_row[10:17]
    cp = a[0] + a[1] * T + a[2] * T ** 2 + a[3] * T ** 3 + a[4] * T ** 4
    h = a[0] + a[1] * T / 2 + a[2] * T ** 2 / 3 + a[3] * T ** 3 / 4 + a[4] * T ** 4 / 5 + a[5] / T
    s = a[0] * np.log(T) + a[1] * T + a[2] * T ** 2 / 2 + a[3] * T ** 3 / 3 + a[4] * T ** 4 / 4 + a[6]
    return cp, h, s


def full_Y(y):
    return np.concatenate([y[1:], [1.0 - y[1:].sum()]])


def mixture(mech, T, P, Y):
    W = mech.W
    S = np.sum(Y / W)
    rho = P / (RU * T * S)
    C = rho * Y / W
    return rho, C


def mixture_h_s(mech, T, P, Y):
    """mass-specific enthalpy (J/kg) and entropy (J/kg/K) of an ideal-gas mixture"""
    h = s = 0.0
    X = (Y / mech.W) / np.sum(Y / mech.W)
    for k in range(mech.ns):
        cp, hk, sk = nasa_eval(mech.nasa[k], T)
        h += Y[k] / mech.W[k] * hk * RU * T
        if Y[k] > 0:
            s += Y[k] / mech.W[k] * RU * (sk - np.log(X[k] * P / PATM))
    return h, s


def tiny_mechanism(names, W, nasa_a, reactions, rtype=None, fall=None, eff=None):
    """Build a Mechanism by hand. nasa_a: [ns, 7] (same set in both ranges)."""
    ns, nr = len(names), len(reactions)
    nasa = np.zeros((ns, 17))
    nasa[:, 0:3] = (200.0, 1000.0, 3500.0)
    nasa[:, 3:10] = nasa_a
    nasa[:, 10:17] = nasa_a
    reac = -np.ones((nr, 3), dtype=np.int64)
    prod = -np.ones((nr, 3), dtype=np.int64)
    arrh = np.zeros((nr, 3))
    for i, (r, p, ar) in enumerate(reactions):
        reac[i, : len(r)] = r
        prod[i, : len(p)] = p
        arrh[i] = ar
    return synth.Mechanism(
        name="tiny", ns=ns, nr=nr, names=list(names), elements=["X"],
        comp=np.ones((ns, 1), dtype=np.int64), W=np.asarray(W, float), nasa=nasa,
        reac=reac, prod=prod, arrh=arrh,
        rtype=np.zeros(nr, dtype=np.int64) if rtype is None else np.asarray(rtype),
        eff=np.ones((nr, ns)) if eff is None else eff,
        fall=np.zeros((nr, 7)) if fall is None else fall)


# ----------------------------------------------------------------------------
# thermo
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["h2", "ch4"])
@pytest.mark.parametrize("T", [450.0, 998.0, 1003.0, 1800.0, 3100.0])
def test_thermo_identities(kind, T, h2_mech, ch4_mech):
    mech = h2_mech if kind == "h2" else ch4_mech
    cp, h, s = O.thermo(mech, T)
    e = 1e-3
    cpp, hp, sp = O.thermo(mech, T + e)
    cpm, hm, sm = O.thermo(mech, T - e)
    dhdT = ((T + e) * hp - (T - e) * hm) / (2 * e)     # d(h/R)/dT = cp/R
    dsdT = (sp - sm) / (2 * e)                         # d(s/R)/dT = cp/(R T)
    np.testing.assert_allclose(dhdT, cp, rtol=1e-8)
    np.testing.assert_allclose(dsdT, cp / T, rtol=1e-7)
    assert np.all(cp >= 2.5 - 1e-9) and np.all(cp <= 6.0 + 1e-9)


def test_thermo_selects_range_by_T_mid(h2_mech):
    mech = copy.deepcopy(h2_mech)
    mech.nasa[:, 10:17] = mech.nasa[:, 3:10] * 1.5      # a different high-T set
    for T in (700.0, 999.999, 1000.0, 1500.0):
        cp, h, s = O.thermo(mech, T)
        for k in range(mech.ns):
            want = nasa_eval(mech.nasa[k], T)
            np.testing.assert_allclose([cp[k], h[k], s[k]], want, rtol=1e-13)
    cp_lo, _, _ = O.thermo(mech, 999.0)
    cp_hi, _, _ = O.thermo(mech, 1001.0)
    assert np.all(cp_hi > 1.3 * cp_lo)


# ----------------------------------------------------------------------------
# rates: closed forms
# ----------------------------------------------------------------------------

def _ab_mech(kf=1e5, ds=1.0):
    a = np.zeros((3, 7))
    a[:, 0] = 3.5
    a[1, 6] = ds                      # s_B/R - s_A/R = ds, equal enthalpies
    return tiny_mechanism(["A", "B", "I"], [30.0, 30.0, 28.0], a,
                          [([0], [1], (kf, 0.0, 0.0))])


def test_isothermal_A_to_B_closed_form():
    kf, ds = 1e5, 1.0
    mech = _ab_mech(kf, ds)
    kr = kf / np.exp(ds)              # Kc = Kp = exp(ds) for sum(nu) = 0, dh = 0
    T0, P = 1000.0, 2.0 * PATM
    YA0, YB0 = 0.3, 0.1
    y0 = np.array([T0, YA0, YB0])
    # source term against mass action
    f, rc = O.rhs(mech, P, y0)
    Y = full_Y(y0)
    rho, C = mixture(mech, T0, P, Y)
    q = kf * C[0] - kr * C[1]
    np.testing.assert_allclose(f[1], -30.0 * q / rho, rtol=1e-13)
    np.testing.assert_allclose(f[2], 30.0 * q / rho, rtol=1e-13)
    assert abs(f[0]) < 1e-9 * abs(f[1])
    # trajectory against the closed form
    Yeq = kr / (kf + kr) * (YA0 + YB0)
    om = O.OracleMech(mech)
    for t in (1e-6, 1e-5, 5e-5):
        st = synth.States(Y=np.array([[YA0], [YB0], [0.6]]), T=np.array([T0]), P=np.array([P]))
        Yo, To, cnt = O.integrate(om, st, t, rtol=1e-12, atol=1e-20)
        want = Yeq + (YA0 - Yeq) * np.exp(-(kf + kr) * t)
        np.testing.assert_allclose(Yo[0, 0], want, rtol=1e-9)
        np.testing.assert_allclose(Yo[1, 0], YA0 + YB0 - want, rtol=1e-9)
        np.testing.assert_allclose(To[0], T0, rtol=1e-12)
        assert cnt[0, 7] == 0


def test_reverse_rate_uses_pressure_factor_for_nonzero_sum_nu():
    """A <-> 2B: Kc = Kp (Patm/(Ru T))^1 with Kp from the Gibbs energies."""
    a = np.zeros((3, 7))
    a[:, 0] = 3.5
    a[1, 5] = 2000.0
    a[1, 6] = 3.0
    mech = tiny_mechanism(["A", "B", "I"], [30.0, 15.0, 28.0], a, [([0], [1, 1], (1e4, 0.5, 800.0))])
    T = 1400.0
    C = np.array([0.01, 0.003, 0.05])
    kf_eff, kr_eff = O.rate_constants(mech, T, C)
    kf = 1e4 * T ** 0.5 * np.exp(-800.0 / T)
    g = [nasa_eval(mech.nasa[k], T) for k in range(3)]
    lnKp = 2 * (g[1][2] - g[1][1]) - (g[0][2] - g[0][1])
    Kc = np.exp(lnKp) * PATM / (RU * T)
    np.testing.assert_allclose(kf_eff[0], kf, rtol=1e-13)
    np.testing.assert_allclose(kr_eff[0], kf / Kc, rtol=1e-12)


def _troe_mech():
    a = np.zeros((4, 7))
    a[:, 0] = 3.5
    fall = np.zeros((1, 7))
    fall[0] = (1e9, -1.0, 300.0, 0.6, 200.0, 1500.0, 5000.0)
    eff = np.ones((1, 4))
    eff[0, 0] = 2.5
    return tiny_mechanism(["A", "B", "AB", "I"], [10.0, 20.0, 30.0, 28.0], a,
                          [([0, 1], [2], (3e8, 0.3, 100.0))], rtype=[2], fall=fall, eff=eff)


def test_troe_factor_at_center_and_limits():
    mech = _troe_mech()
    T = 1300.0
    a, T3, T1, T2 = 0.6, 200.0, 1500.0, 5000.0
    Fc = (1 - a) * np.exp(-T / T3) + a * np.exp(-T / T1) + np.exp(-T2 / T)
    c = -0.4 - 0.67 * np.log10(Fc)
    k0 = 1e9 * T ** -1.0 * np.exp(-300.0 / T)
    kinf = 3e8 * T ** 0.3 * np.exp(-100.0 / T)
    # [M] = eff . C: put the collider in the inert only
    def kf_at(M):
        C = np.array([0.0, 0.0, 0.0, M])
        return O.rate_constants(mech, T, C)[0][0]
    Pr_c = 10.0 ** (-c)
    Mc = Pr_c * kinf / k0
    np.testing.assert_allclose(kf_at(Mc), kinf * Pr_c / (1 + Pr_c) * Fc, rtol=1e-12)
    # both limits approach Fcent^(d^2/(1+d^2)) (X -> -1/d); F stays in [Fcent, 1]
    F_lim = Fc ** (0.14 ** 2 / (1 + 0.14 ** 2))
    M_lo, M_hi = Mc * 1e-250, Mc * 1e250
    r_lo = kf_at(M_lo) / (k0 * M_lo)
    r_hi = kf_at(M_hi) / kinf
    for r in (r_lo, r_hi):
        assert Fc <= r <= 1.0
        assert abs(r / F_lim - 1) < 5e-3     # approached like 1/log(Pr)
    # efficiencies enter [M]: C_A weighted by 2.5
    C = np.array([0.004, 0.0, 0.0, 0.0])
    np.testing.assert_allclose(O.rate_constants(mech, T, C)[0][0], kf_at(0.01), rtol=1e-13)
    # falloff factor increases with [M]
    Ms = Mc * np.logspace(-4, 4, 9)
    ks = [kf_at(M) for M in Ms]
    assert np.all(np.diff(ks) > 0)


def test_third_body_scales_with_M(h2_mech):
    mech = h2_mech
    i = int(np.where(mech.rtype == 1)[0][0])
    T = 1500.0
    C = np.full(mech.ns, 1e-3)
    kf1, kr1 = O.rate_constants(mech, T, C)
    kf2, kr2 = O.rate_constants(mech, T, 3 * C)
    np.testing.assert_allclose(kf2[i], 3 * kf1[i], rtol=1e-13)
    np.testing.assert_allclose(kr2[i], 3 * kr1[i], rtol=1e-13)
    e = np.where(mech.rtype == 0)[0][0]
    np.testing.assert_allclose(kf2[e], kf1[e], rtol=1e-15)


# ----------------------------------------------------------------------------
# Jacobians
# ----------------------------------------------------------------------------

def _fd4(f, y, j, e):
    yp, ym, yp2, ym2 = y.copy(), y.copy(), y.copy(), y.copy()
    yp[j] += e
    ym[j] -= e
    yp2[j] += 2 * e
    ym2[j] -= 2 * e
    return (8 * (f(yp) - f(ym)) - (f(yp2) - f(ym2))) / (12 * e)


@pytest.mark.parametrize("kind,n", [("h2", 12), ("ch4", 4)])
def test_analytical_jacobian_against_central_differences(kind, n, h2_mech, ch4_mech):
    mech = h2_mech if kind == "h2" else ch4_mech
    om = O.OracleMech(mech)
    st = synth.make_states(mech, n, seed=7, T_range=(800.0, 2600.0))
    y = O.state_vector(st)
    worst = 0.0
    for i in range(n):
        yi, P = y[:, i].copy(), st.P[i]
        J, rc = O.jac(om, P, yi)
        assert rc == 0
        f = lambda v: O.rhs(om, P, v)[0]
        for j in range(mech.ns):
            colmax = np.abs(J[:, j]).max() + 1e-300
            best = np.inf
            scale = yi[0] if j == 0 else max(abs(yi[j]), 1e-3)
            for rel in (1e-3, 3e-4, 1e-4, 3e-5, 1e-5):
                d = _fd4(f, yi, j, rel * scale)
                best = min(best, np.abs(d - J[:, j]).max() / colmax)
            worst = max(worst, best)
    assert worst < 2e-6, worst


def test_fd_jacobian_follows_cvode_increment_rule(h2_mech):
    """The difference-quotient Jacobian is defined by its increment rule
    (CVODE's dense DQ Jacobian): inc_j = max(sqrt(eps)|y_j|, minInc / w_j),
    minInc = 1000 |h| eps N ||f0||_w (1 if the norm is 0), w_j = 1/scal_j.
    Column j must be (f(y + inc_j e_j) - f(y)) / inc_j; and where the analytical
    column stands well above the cancellation noise of f the two agree."""
    om = O.OracleMech(h2_mech)
    st = synth.make_states(h2_mech, 6, seed=11)
    y = O.state_vector(st)
    eps = np.finfo(float).eps
    n_close = 0
    for i in range(6):
        yi, P = y[:, i].copy(), st.P[i]
        f0, _ = O.rhs(om, P, yi)
        scal = 1e-9 + 1e-5 * np.abs(yi)
        J, _ = O.jac(om, P, yi)
        for h in (1e-14, 1e-8):
            Jfd, rc = O.jac_fd(om, P, yi, f0, h, scal)
            assert rc == 0
            fn = np.sqrt(np.mean((f0 / scal) ** 2))
            min_inc = 1000.0 * h * eps * len(yi) * fn if fn > 0 else 1.0
            for j in range(len(yi)):
                inc = max(np.sqrt(eps) * abs(yi[j]), min_inc * scal[j])
                yp = yi.copy()
                yp[j] += inc
                col = (O.rhs(om, P, yp)[0] - f0) / inc
                np.testing.assert_allclose(Jfd[:, j], col, rtol=1e-12, atol=0)
            err = np.abs(Jfd - J).max(axis=0) / (np.abs(J).max(axis=0) + 1e-300)
            n_close += int(np.sum(err < 1e-2))
    # about 60 % of the columns sit above the noise on these states (zero species do not)
    assert n_close >= 0.5 * 6 * 2 * h2_mech.ns, n_close


# ----------------------------------------------------------------------------
# integrations: invariants
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("kind,n,dt", [("h2", 64, 1e-4), ("ch4", 8, 1e-5)])
def test_conservation_along_integration(kind, n, dt, h2_mech, ch4_mech):
    mech = h2_mech if kind == "h2" else ch4_mech
    st = synth.make_states(mech, n, seed=5, T_range=(900.0, 2500.0))
    Y, T, cnt = O.integrate(mech, st, dt)
    assert np.all(cnt[:, 7] == 0)
    # elements (kmol per kg) are a linear invariant of the ODE
    el0 = (mech.comp.T.astype(float) / mech.W[None, :]) @ st.Y
    el1 = (mech.comp.T.astype(float) / mech.W[None, :]) @ Y
    np.testing.assert_allclose(el1, el0, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(Y.sum(axis=0), 1.0, rtol=0, atol=1e-14)
    assert np.all((T > 300) & (T < 4000))
    for i in range(n):
        h0, s0 = mixture_h_s(mech, st.T[i], st.P[i], st.Y[:, i])
        h1, s1 = mixture_h_s(mech, T[i], st.P[i], Y[:, i])
        cp_scale = 1500.0 * T[i]
        assert abs(h1 - h0) < 2e-5 * cp_scale, (i, h0, h1)
        assert s1 >= s0 - 1e-6 * abs(s0), (i, s0, s1)   # second law, adiabatic isobaric


def test_entropy_never_decreases_along_trajectory(h2_mech):
    st = synth.make_states(h2_mech, 4, seed=8, T_range=(1000.0, 1400.0))
    om = O.OracleMech(h2_mech)
    for i in range(4):
        s_prev = -np.inf
        for t in (1e-7, 1e-6, 1e-5, 1e-4, 1e-3):
            Y, T, cnt = O.integrate(om, st.subset([i]), t)
            _, s = mixture_h_s(h2_mech, T[0], st.P[i], Y[:, 0])
            assert s >= s_prev - 1e-9 * abs(s)
            s_prev = s


def test_detailed_balance_at_equilibrium(h2_mech):
    """After a long time every reaction quotient equals Kc from Gibbs energies.
    (The slowest synthetic reactions have time scales up to ~1e5 s, hence
    the 1e6 s horizon; Radau's step grows geometrically near equilibrium.)"""
    mech = h2_mech
    st = synth.make_states(mech, 3, seed=9, T_range=(1500.0, 2200.0))
    Y, T, cnt = O.integrate(mech, st, 1e6)
    assert np.all(cnt[:, 7] == 0)
    for i in range(3):
        rho, C = mixture(mech, T[i], st.P[i], Y[:, i])
        g = np.array([nasa_eval(mech.nasa[k], T[i]) for k in range(mech.ns)])
        checked = 0
        for r in range(mech.nr):
            re = [k for k in mech.reac[r] if k >= 0]
            pr = [k for k in mech.prod[r] if k >= 0]
            if min(C[re + pr]) < 1e-25:
                continue
            lnQ = np.sum(np.log(C[pr])) - np.sum(np.log(C[re]))
            dnu = len(pr) - len(re)
            lnKc = (sum(g[k, 2] - g[k, 1] for k in pr) - sum(g[k, 2] - g[k, 1] for k in re)
                    + dnu * np.log(PATM / (RU * T[i])))
            assert abs(lnQ - lnKc) < 1e-6, (r, lnQ, lnKc)
            checked += 1
        assert checked >= mech.nr // 2
        f, _ = O.rhs(mech, st.P[i], np.concatenate([[T[i]], Y[:-1, i]]))
        assert abs(f[0]) < 1e-3          # K/s: at rest


def test_batch_is_independent_of_thread_count(h2_mech):
    st = synth.make_states(h2_mech, 48, seed=12)
    a = O.integrate(h2_mech, st, 1e-5, nthreads=1)
    b = O.integrate(h2_mech, st, 1e-5, nthreads=4)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    cnt = a[2]
    assert np.all(cnt[:, 1] + (cnt[:, 0] - cnt[:, 1]) == cnt[:, 0])
    assert np.all(cnt[:, 2] <= cnt[:, 0] - cnt[:, 1])
    assert np.all(cnt[:, 6] >= cnt[:, 1])


def test_error_norm_and_divergence_measures():
    y = np.ones((3, 2))
    yt = np.ones((3, 2))
    yt[0, 1] = 1.0 + 1e-6
    E = O.error_norm(y, yt, atol=1e-10, rtol=1e-6)
    assert E[0] == 0.0
    np.testing.assert_allclose(E[1], np.sqrt(((1e-6 / (1e-10 + 1e-6 * (1 + 1e-6))) ** 2) / 3))
    assert O.divergence(np.full(64, 7))[0] == 0.0
    d = np.zeros(32)
    d[3] = 10
    np.testing.assert_allclose(O.divergence(d)[0], 1 - 1 / 32)
