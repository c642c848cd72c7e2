"""The seeded input generator: sizes, reaction types, element balance,
reproducibility and the composition recipe."""
import numpy as np
import pytest

from paper_1607_03884_gb300 import synth


@pytest.mark.parametrize("kind,ns,nr,ntb,ntroe", [("h2", 13, 27, 5, 1), ("ch4", 53, 325, 30, 15)])
def test_mechanism_sizes_and_balance(kind, ns, nr, ntb, ntroe, h2_mech, ch4_mech):
    m = h2_mech if kind == "h2" else ch4_mech
    assert (m.ns, m.nr) == (ns, nr)
    assert int(np.sum(m.rtype == 1)) == ntb and int(np.sum(m.rtype == 2)) == ntroe
    for i in range(m.nr):
        r = [k for k in m.reac[i] if k >= 0]
        p = [k for k in m.prod[i] if k >= 0]
        np.testing.assert_array_equal(m.comp[r].sum(axis=0), m.comp[p].sum(axis=0))
        assert m.ns - 1 not in r + p                # the inert only collides
        assert 1 <= len(r) <= 3 and 1 <= len(p) <= 3
    used = set(m.reac[m.reac >= 0]) | set(m.prod[m.prod >= 0])
    assert used == set(range(m.ns - 1))
    assert np.all(m.arrh[:, 0] > 0)
    assert np.all(m.W > 0)


def test_mechanism_is_reproducible():
    a = synth.make_mechanism("h2")
    b = synth.make_mechanism("h2")
    for f in ("W", "nasa", "reac", "prod", "arrh", "rtype", "eff", "fall"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    c = synth.make_mechanism("h2", seed=7)
    assert not np.array_equal(a.arrh, c.arrh)


def test_states_recipe(h2_mech):
    st = synth.make_states(h2_mech, 4096, seed=1, mode="mixed")
    np.testing.assert_allclose(st.Y.sum(axis=0), 1.0, atol=1e-15)
    assert np.all(st.Y >= 0)
    hot = st.T >= 1800.0
    assert 0.15 < hot.mean() < 0.25
    assert np.all((st.T[~hot] >= 900) & (st.T[~hot] <= 1200))
    assert np.all((st.P >= 101325.0) & (st.P <= 25 * 101325.0))
    st2 = synth.make_states(h2_mech, 4096, seed=1, mode="mixed")
    np.testing.assert_array_equal(st.Y, st2.Y)
    yu, yb = synth.fuel_air_and_products(h2_mech)
    # stoichiometric H2/air: element H / element O ratio 2:1 in both
    el = h2_mech.comp.T.astype(float) @ (yu / h2_mech.W)
    eb = h2_mech.comp.T.astype(float) @ (yb / h2_mech.W)
    np.testing.assert_allclose(el, eb, rtol=1e-12)
    assert abs(el[0] / el[1] - 2.0) < 1e-12


@pytest.mark.parametrize("name,kind,n,seed", [
    ("h2_1024", "h2", 1024, 42), ("h2_mixed_2p20", "h2", 1 << 20, 43),
    ("ch4_2p18", "ch4", 1 << 18, 44), ("ch4_2p16", "ch4", 1 << 16, 45),
    ("ch4_learned_test_2p20", "ch4", 1 << 20, 46), ("ch4_learned_train_2p20", "ch4", 1 << 20, 47)])
def test_workload_registry(name, kind, n, seed):
    w = synth.WORKLOADS[name]
    assert (w["kind"], w["n"], w["seed"]) == (kind, n, seed)
    if n <= 1 << 16:   # a prefix is the first states of the full batch
        mech, full, _ = synth.workload(name)
        _, pre, _ = synth.workload(name, 16)
        np.testing.assert_array_equal(pre.T, full.T[:16])
        np.testing.assert_array_equal(pre.Y, full.Y[:, :16])


@pytest.mark.parametrize("kind", ["h2", "ch4"])
def test_thermo_fits_are_monotone_in_range(kind, h2_mech, ch4_mech):
    """cp/R of every species is monotone in T and within [2.5, 6] over
    300-3000 K, with the same coefficients in both NASA-7 ranges."""
    m = h2_mech if kind == "h2" else ch4_mech
    T = np.linspace(300.0, 3000.0, 271)
    for k in range(m.ns):
        lo, hi = m.nasa[k, 3:10], m.nasa[k, 10:17]
        np.testing.assert_array_equal(lo, hi)
        cp = lo[0] + T * (lo[1] + T * (lo[2] + T * (lo[3] + T * lo[4])))
        assert np.all(np.diff(cp) >= -1e-12), k
        assert cp.min() >= 2.5 - 1e-9 and cp.max() <= 6.0 + 1e-9, (k, cp.min(), cp.max())


def test_structure_of_a_concentration_based_jacobian():
    """How sparse the seeded mechanisms' concentration-based Newton matrices
    are (the paper's proposed reformulation, Sec. 3.3 and Sec. 4): in the
    state [T, V, n_0 .. n_{ns-2}] (extensive moles, constant pressure, inert
    bath of efficiency 1) two species are coupled only through a shared
    reaction or a non-default collision efficiency, with full T and V rows
    and columns.  The seeded mechanisms pair species at random, so the
    structure is dense: the 13-species one fills 97 % of its 14 x 14
    matrix, the 53-species one 74 % of 54 x 54, and an LU in a minimum-
    degree order (scipy's, here) fills 90 % or more.  The sparse LU's saving
    is therefore in its first pivots (a sixth of the factorisation's
    operations on CH4)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    dens = {}
    for kind in ("h2", "ch4"):
        m = synth.make_mechanism(kind)
        ns, inert = m.ns, m.ns - 1
        N = ns + 1
        S = np.eye(N, dtype=bool)
        S[:2, :] = True
        S[:, :2] = True
        for i in range(m.nr):
            sps = {int(x) for x in m.reac[i] if x >= 0} | {int(x) for x in m.prod[i] if x >= 0}
            cols = set(sps)
            if m.rtype[i]:
                assert m.eff[i][inert] == 1.0
                cols |= {int(k) for k in np.where(m.eff[i] != 1.0)[0]}
            for r in sps - {inert}:
                for c in cols - {inert}:
                    S[2 + r, 2 + c] = True
        A = sp.csc_matrix(S.astype(float) + N * np.eye(N))
        lu = spl.splu(A, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                      options=dict(SymmetricMode=True))
        dens[kind] = (S.mean(), (lu.L.nnz + lu.U.nnz - N) / N / N)
    print("\nconcentration-based Newton matrix: density, LU fill:", dens)
    assert dens["h2"][0] > 0.9 and dens["ch4"][0] > 0.6
    assert dens["ch4"][1] > 0.85
