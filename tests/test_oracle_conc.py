"""Pins of the oracle's concentration-based form (chem.c orc_rhs_conc /
orc_jac_conc, batch.c form 1): the reformulation the paper proposes for a
sparse Jacobian (Sec. 3.3, Sec. 4).

What pins what:
* Right-hand side: it is the mass-fraction reactor's (already pinned) in
  other variables.  dT/dt is the same; W_k dn_k/dt = dY_k/dt per unit mass;
  dV/dt is the time derivative of 1/rho = Ru T sum(Y_k/W_k)/P, written here
  from the mass-fraction rates.
* Jacobian: against a fourth-order central difference of the right-hand
  side (best agreement over a sweep of increments), and its structure: an
  entry between two species is exactly zero unless they share a reaction
  or one is a collider with a non-default efficiency in a reaction of the
  other.
* Integrations: the same solution as the mass-fraction form at tight
  tolerances (one reactor, two state vectors), conservation of element
  moles (a linear invariant of dn/dt = V wdot that every RK method keeps),
  and the conversions to and from phi.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1607_03884_gb300 import synth

RU = 8314.46261815324


def _fd4(f, y, j, e):
    yp, ym, yp2, ym2 = y.copy(), y.copy(), y.copy(), y.copy()
    yp[j] += e
    ym[j] -= e
    yp2[j] += 2 * e
    ym2[j] -= 2 * e
    return (8 * (f(yp) - f(ym)) - (f(yp2) - f(ym2))) / (12 * e)


def structure(mech):
    """Boolean (ns+1) x (ns+1) pattern of the concentration-based Jacobian
    in phi order [T, V, n_0..n_{ns-2}], from the reaction lists."""
    ns, inert = mech.ns, mech.ns - 1
    N = ns + 1
    S = np.eye(N, dtype=bool)
    S[:2, :] = True
    S[:, :2] = True
    for i in range(mech.nr):
        sps = {int(x) for x in mech.reac[i] if x >= 0} | {int(x) for x in mech.prod[i] if x >= 0}
        cols = set(sps)
        if mech.rtype[i]:
            cols |= {int(k) for k in np.where(mech.eff[i] != mech.eff[i][inert])[0]}
        for r in sps - {inert}:
            for c in cols - {inert}:
                S[2 + r, 2 + c] = True
    return S


@pytest.mark.parametrize("kind", ["h2", "ch4"])
def test_conc_rhs_is_the_mass_fraction_rhs(kind):
    mech = synth.make_mechanism(kind)
    st = synth.make_states(mech, 6, seed=11, T_range=(800.0, 2600.0))
    W = mech.W
    for i in range(st.n):
        Y, T, P = st.Y[:, i], st.T[i], st.P[i]
        phi = O.to_conc(mech, Y, T, P)
        f, rc = O.rhs_conc(mech, P, phi)
        assert rc == 0
        fy, rc = O.rhs(mech, P, np.concatenate([[T], Y[:-1]]))
        assert rc == 0
        assert abs(f[0] - fy[0]) <= 1e-12 * abs(fy[0]) + 1e-300
        dY = fy[1:]
        scale = np.abs(dY).max()
        assert np.abs(W[:-1] * f[2:] - dY).max() <= 1e-12 * scale
        # d(1/rho)/dt from the mass-fraction rates; the inert's is minus the sum
        dYall = np.concatenate([dY, [-dY.sum()]])
        dV = RU / P * (np.sum(Y / W) * fy[0] + T * np.sum(dYall / W))
        assert abs(f[1] - dV) <= 1e-10 * (abs(dV) + RU * T * np.sum(Y / W) / P * 1e-12), (f[1], dV)


@pytest.mark.parametrize("kind,n", [("h2", 8), ("ch4", 3)])
def test_conc_jacobian_against_central_differences(kind, n):
    mech = synth.make_mechanism(kind)
    om = O.OracleMech(mech)
    st = synth.make_states(mech, n, seed=7, T_range=(800.0, 2600.0))
    worst = 0.0
    for i in range(n):
        P = st.P[i]
        phi = O.to_conc(mech, st.Y[:, i], st.T[i], P)
        J, rc = O.jac_conc(om, P, phi)
        assert rc == 0
        f = lambda v: O.rhs_conc(om, P, v)[0]
        for j in range(mech.ns + 1):
            colmax = np.abs(J[:, j]).max() + 1e-300
            best = np.inf
            scale = abs(phi[j]) if j < 2 else max(abs(phi[j]), 1e-5)
            for rel in (1e-3, 3e-4, 1e-4, 3e-5, 1e-5):
                d = _fd4(f, phi, j, rel * scale)
                best = min(best, np.abs(d - J[:, j]).max() / colmax)
            worst = max(worst, best)
    assert worst < 2e-6, worst


@pytest.mark.parametrize("kind", ["h2", "ch4"])
def test_conc_jacobian_structure(kind):
    """Species entries outside the reaction structure are exactly zero; the
    structure is what makes the form sparse."""
    mech = synth.make_mechanism(kind)
    S = structure(mech)
    st = synth.make_states(mech, 4, seed=5, T_range=(800.0, 2600.0))
    seen = np.zeros_like(S)
    for i in range(st.n):
        phi = O.to_conc(mech, st.Y[:, i], st.T[i], st.P[i])
        J, rc = O.jac_conc(mech, st.P[i], phi)
        assert rc == 0
        assert np.all(J[~S] == 0.0)
        seen |= J != 0.0
    # the pattern is not loose: almost every structural entry is non-zero
    assert seen[S].mean() > 0.9
    if kind == "ch4":
        assert S.mean() < 0.8


@pytest.mark.parametrize("kind,dt", [("h2", 1e-6), ("h2", 1e-4), ("ch4", 1e-6), ("ch4", 1e-4)])
def test_conc_integration_matches_the_mass_fraction_form(kind, dt):
    """One reactor, two state vectors: at tight tolerances both forms reach
    the same (Y, T) after dt."""
    mech = synth.make_mechanism(kind)
    n = 12 if kind == "h2" else 3
    st = synth.make_states(mech, n, seed=21, mode="mixed" if kind == "h2" else "correlated")
    kw = dict(rtol=1e-11, atol=1e-20, transform_tol=False)
    Ya, Ta, ca = O.integrate(mech, st, dt, **kw)
    Yb, Tb, cb = O.integrate(mech, st, dt, form="conc", **kw)
    assert np.all(ca[:, 7] == 0) and np.all(cb[:, 7] == 0)
    ya = np.concatenate([Ta[None], Ya[:-1]])
    yb = np.concatenate([Tb[None], Yb[:-1]])
    E = O.error_norm(yb, ya)
    assert E.max() < 1e-6, E
    assert np.abs(Yb.sum(axis=0) - 1.0).max() < 1e-13


def test_conc_integration_conserves_element_moles():
    """sum_k comp[k, e] n_k over the active species is a linear invariant of
    dn_k/dt = V wdot_k (the bath gas takes part in no reaction), so Radau
    keeps it to rounding.  The mixture's mass is not linear in phi (the bath
    gas's moles follow from V and T): it moves with the integration error,
    and the outputs are normalised by it."""
    mech = synth.make_mechanism("ch4")
    om = O.OracleMech(mech)
    st = synth.make_states(mech, 3, seed=22)
    comp = np.asarray(mech.comp, dtype=np.float64)[:-1]
    for i in range(st.n):
        P = st.P[i]
        phi0 = O.to_conc(mech, st.Y[:, i], st.T[i], P)
        phi, stats = O.radau(lambda t, v: O.rhs_conc(om, P, v)[0],
                             lambda t, v: O.jac_conc(om, P, v)[0], phi0, 0.0, 1e-4)
        assert stats["status"] == 0
        e0, e1 = comp.T @ phi0[2:], comp.T @ phi[2:]
        assert np.abs(e1 - e0).max() <= 1e-13 * np.abs(e0).max(), (e0, e1)
        nin = P * phi[1] / (RU * phi[0]) - phi[2:].sum()
        mass = mech.W[:-1] @ phi[2:] + mech.W[-1] * nin
        assert abs(mass - 1.0) < 1e-4


def test_conc_conversions_round_trip():
    mech = synth.make_mechanism("ch4")
    st = synth.make_states(mech, 5, seed=23)
    phi = O.to_conc(mech, st.Y, st.T, st.P)
    assert phi.shape == (mech.ns + 1, st.n)
    rho = st.P / (RU * st.T * np.sum(st.Y / mech.W[:, None], axis=0))
    np.testing.assert_allclose(phi[1], 1.0 / rho, rtol=1e-14)
    Y, T = O.from_conc(mech, phi, st.P)
    np.testing.assert_array_equal(T, st.T)
    np.testing.assert_allclose(Y, st.Y, rtol=1e-13, atol=1e-17)


def test_per_component_atol_is_a_change_of_variables():
    """orc_opts.atol_scale (the moles' atol / W_k of the concentration form):
    Radau with weights atol s_i + rtol |y_i| is Radau on z = y / s with the
    scalar atol (the method is invariant under the scaling, and so are its
    error and Newton norms).  Both runs take the same steps and agree to
    rounding."""
    mech = synth.make_mechanism("h2")
    om = O.OracleMech(mech)
    st = synth.make_states(mech, 2, seed=31, T_range=(1000.0, 1300.0))
    s = np.concatenate([[1.0, 1.0], 1.0 / mech.W[:-1]])
    for i in range(st.n):
        P = st.P[i]
        phi0 = O.to_conc(mech, st.Y[:, i], st.T[i], P)
        f = lambda t, v: O.rhs_conc(om, P, v)[0]
        J = lambda t, v: O.jac_conc(om, P, v)[0]
        ya, sa = O.radau(f, J, phi0, 0.0, 1e-4, atol_scale=s)
        fz = lambda t, z: f(t, z * s) / s
        Jz = lambda t, z: J(t, z * s) * s[None, :] / s[:, None]
        zb, sb = O.radau(fz, Jz, phi0 / s, 0.0, 1e-4)
        assert sa["status"] == 0 and sb["status"] == 0
        assert sa["nstep"] == sb["nstep"] and sa["naccpt"] == sb["naccpt"]
        np.testing.assert_allclose(zb * s, ya, rtol=1e-9, atol=1e-18)
        # and the scaling matters: the scalar atol on the moles takes fewer steps
        yc, sc = O.radau(f, J, phi0, 0.0, 1e-4)
        assert sc["nstep"] < sa["nstep"]
