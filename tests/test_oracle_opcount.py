"""The counted restatement of the path (oracle/opcount.py) evaluates the same
functions as the oracle: its right-hand side and analytical Jacobian equal
orc_rhs and orc_jac on states of both mechanisms (Troe and third-body
reactions included), its LU and solves solve the systems, and its counts
follow the reaction network's structure, not the state."""
import numpy as np
import pytest

from oracle import opcount as OC
from oracle import oracle as O
from paper_1607_03884_gb300 import synth


@pytest.mark.parametrize("kind", ["h2", "ch4"])
def test_counted_rhs_and_jacobian_equal_the_oracle(kind):
    mech = synth.make_mechanism(kind)
    assert np.any(mech.rtype == 2) and np.any(mech.rtype == 1)
    tb = OC.Tables(mech)
    om = O.OracleMech(mech)
    st = synth.make_states(mech, 8, seed=21, T_range=(800.0, 2600.0))
    y = O.state_vector(st)
    counts = set()
    for i in range(st.n):
        yi = [OC.F(v) for v in y[:, i]]
        with OC.counting() as t:
            f, J = OC.evaluate(tb, st.P[i], yi, want_jac=True)
        counts.add(tuple(sorted(t.c.items())))
        fo, _ = O.rhs(om, st.P[i], y[:, i])
        Jo, _ = O.jac(om, st.P[i], y[:, i])
        fv = np.array([float(v) for v in f])
        Jv = np.array([[float(v) for v in r] for r in J])
        np.testing.assert_allclose(fv, fo, rtol=1e-11, atol=1e-13 * np.abs(fo).max())
        colmax = np.abs(Jo).max(axis=0) + 1e-300
        assert np.max(np.abs(Jv - Jo) / colmax) < 1e-10
    assert len(counts) == 1          # the same work at every state


def test_counted_lu_and_solves_solve_the_systems():
    rng = np.random.default_rng(5)
    n = 9
    A = rng.normal(size=(n, n)) + n * np.eye(n) * 0.3
    b = rng.normal(size=n)
    a = [[OC.F(v) for v in row] for row in A]
    piv = OC.lu_real(a)
    x = np.array([float(v) for v in OC.solve_real(a, piv, [OC.F(v) for v in b])])
    np.testing.assert_allclose(A @ x, b, rtol=1e-12, atol=1e-12)
    Ac = A + 1j * rng.normal(size=(n, n))
    bc = rng.normal(size=n) + 1j * rng.normal(size=n)
    ac = [[(OC.F(v.real), OC.F(v.imag)) for v in row] for row in Ac]
    pc = OC.lu_cplx(ac)
    xc = OC.solve_cplx(ac, pc, [(OC.F(v.real), OC.F(v.imag)) for v in bc])
    xc = np.array([float(r) + 1j * float(i) for r, i in xc])
    np.testing.assert_allclose(Ac @ xc, bc, rtol=1e-12, atol=1e-12)


def test_counting_scalar_tallies_each_operation():
    x, y = OC.F(3.0), OC.F(2.0)
    with OC.counting() as t:
        z = (x + y) * x - y / x
        w = -z
        _ = OC.exp(w) + 1.0
    assert (t.c["add"], t.c["mul"], t.c["div"], t.c["exp"]) == (3, 1, 1, 1)
    assert t.flops == 5 and t.transc == 1


@pytest.mark.parametrize("kind", ["h2", "ch4"])
def test_counted_conc_form_equals_the_oracle(kind):
    """evaluate_conc (the counted concentration-based form) equals
    orc_rhs_conc / orc_jac_conc, at the same cost at every state."""
    mech = synth.make_mechanism(kind)
    tb = OC.Tables(mech)
    om = O.OracleMech(mech)
    st = synth.make_states(mech, 6, seed=23, T_range=(800.0, 2600.0))
    counts = set()
    for i in range(st.n):
        phi = O.to_conc(mech, st.Y[:, i], st.T[i], st.P[i])
        np.testing.assert_allclose(OC.conc_state(mech, st.Y[:, i], st.T[i], st.P[i]), phi,
                                   rtol=1e-15)
        with OC.counting() as t:
            f, J = OC.evaluate_conc(tb, st.P[i], [OC.F(v) for v in phi], want_jac=True)
        counts.add(tuple(sorted(t.c.items())))
        fo, _ = O.rhs_conc(om, st.P[i], phi)
        Jo, _ = O.jac_conc(om, st.P[i], phi)
        fv = np.array([float(v) for v in f])
        Jv = np.array([[float(v) for v in r] for r in J])
        np.testing.assert_allclose(fv, fo, rtol=1e-11, atol=1e-13 * np.abs(fo).max())
        colmax = np.abs(Jo).max(axis=0) + 1e-300
        assert np.max(np.abs(Jv - Jo) / colmax) < 1e-10
    assert len(counts) == 1


@pytest.mark.parametrize("kind", ["h2", "ch4"])
def test_sparse_lu_counts_and_the_library_analysis_agree(kind):
    """The counted sparse LU and solves solve the systems and cost their
    closed forms; this module's minimum-degree order and fill (written
    here) are the library's (kin_conc_analyse), whose factorisation count
    takes one reciprocal per pivot instead of a division per multiplier."""
    from paper_1607_03884_gb300 import kin
    mech = synth.make_mechanism(kind)
    var, pat = OC.conc_structure(mech)
    lvar, lpat, lcnt = kin.conc_analyse(mech)
    assert list(lvar) == var
    np.testing.assert_array_equal(lpat, pat)
    N = pat.shape[0]
    cf = OC.sparse_closed_forms(pat)
    assert lcnt[2] == cf["lu_real"] + N and lcnt[3] == cf["solve_real"]
    rng = np.random.default_rng(8)
    A = np.where(pat, rng.normal(size=(N, N)), 0.0) + N * np.eye(N)
    b = rng.normal(size=N)
    with OC.counting() as t:
        a = [[OC.F(v) for v in row] for row in A]
        OC.lu_sparse_real(a, pat)
    assert t.flops == cf["lu_real"]
    with OC.counting() as t:
        x = OC.solve_sparse_real(a, pat, [OC.F(v) for v in b])
    assert t.flops == cf["solve_real"]
    np.testing.assert_allclose(A @ np.array([float(v) for v in x]), b, rtol=1e-10, atol=1e-10)
    Ac = A + 0.5j * np.where(pat, A, 0.0)
    bc = b - 1j * b
    with OC.counting() as t:
        ac = [[(OC.F(v.real), OC.F(v.imag)) for v in row] for row in Ac]
        OC.lu_sparse_cplx(ac, pat)
    assert t.flops == cf["lu_cplx"]
    with OC.counting() as t:
        xc = OC.solve_sparse_cplx(ac, pat, [(OC.F(v.real), OC.F(v.imag)) for v in bc])
    assert t.flops == cf["solve_cplx"]
    xv = np.array([float(r) + 1j * float(i) for r, i in xc])
    np.testing.assert_allclose(Ac @ xv, bc, rtol=1e-10, atol=1e-10)
