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
