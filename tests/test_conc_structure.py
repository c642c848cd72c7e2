"""The library's symbolic analysis for the concentration-based form's sparse
LU (kin_conc_analyse, host only, no GPU), checked against what the
mathematics fixes: the filled pattern of Gaussian elimination without
pivoting in the returned order (brute force here), a numerical LU of a
matrix with J's pattern that stays inside it, the operation counts
recomputed from the pattern, the minimum-degree choice of the first pivot,
and the oracle's Jacobian vanishing outside the pattern."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1607_03884_gb300 import kin, synth


def j_pattern(mech):
    """J's structure in phi order [T, V, n_0..n_{ns-2}] from the reaction lists."""
    ns, inert = mech.ns, mech.ns - 1
    N = ns + 1
    S = np.eye(N, dtype=bool)
    S[:2, :] = True
    S[:, :2] = True
    for i in range(mech.nr):
        sps = {int(x) for x in mech.reac[i] if x >= 0} | {int(x) for x in mech.prod[i] if x >= 0}
        cols = set(sps)
        if mech.rtype[i]:
            cols |= {int(k) for k in np.where(mech.eff[i] != 1.0)[0]}
        for r in sps:
            for c in cols - {inert}:
                S[2 + r, 2 + c] = True
    return S


def brute_fill(P):
    P = P.copy()
    N = P.shape[0]
    for k in range(N):
        for i in range(k + 1, N):
            if P[i, k]:
                P[i, k + 1:] |= P[k, k + 1:]
    return P


@pytest.mark.parametrize("kind", ["h2", "ch4"])
def test_order_and_fill_are_those_of_elimination(kind):
    mech = synth.make_mechanism(kind)
    var, pat, cnt = kin.conc_analyse(mech)
    N = mech.ns + 1
    assert sorted(var.tolist()) == list(range(N))
    assert var[-2] == 0 and var[-1] == 1          # T and V last
    S = j_pattern(mech)
    Sp = S[np.ix_(var, var)]
    np.testing.assert_array_equal(pat, brute_fill(Sp))
    assert np.all(pat[Sp])
    assert cnt[0] == S.sum() and cnt[1] == pat.sum()
    # operation counts recomputed from the pattern
    lu, sol = 0, N
    for k in range(N):
        l = int(pat[k + 1:, k].sum())
        u = int(pat[k, k + 1:].sum())
        lu += 1 + l + 2 * l * u
        sol += 2 * l + 2 * int(pat[:k, k].sum())
    assert cnt[2] == lu and cnt[3] == sol
    assert lu < 2 * N ** 3 / 3 + N ** 2


@pytest.mark.parametrize("kind", ["h2", "ch4"])
def test_numerical_lu_stays_in_the_pattern(kind):
    """A diagonally dominant matrix with J's pattern, permuted, factorised
    without pivoting: every non-zero of L and U is inside the pattern."""
    mech = synth.make_mechanism(kind)
    var, pat, _ = kin.conc_analyse(mech)
    S = j_pattern(mech)[np.ix_(var, var)]
    N = S.shape[0]
    rng = np.random.default_rng(3)
    A = np.where(S, rng.uniform(-1.0, 1.0, (N, N)), 0.0) + N * np.eye(N)
    for k in range(N):
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    assert np.all(A[~pat] == 0.0)


def test_first_pivot_has_minimum_degree():
    mech = synth.make_mechanism("ch4")
    var, _, _ = kin.conc_analyse(mech)
    S = j_pattern(mech)[2:, 2:]
    G = (S | S.T) & ~np.eye(S.shape[0], dtype=bool)
    deg = G.sum(axis=1)
    first = var[0] - 2
    assert deg[first] == deg.min() and first == int(np.argmin(deg))


@pytest.mark.parametrize("kind", ["h2", "ch4"])
def test_oracle_jacobian_vanishes_outside_the_pattern(kind):
    mech = synth.make_mechanism(kind)
    var, pat, _ = kin.conc_analyse(mech)
    st = synth.make_states(mech, 3, seed=9, T_range=(900.0, 2400.0))
    for i in range(st.n):
        phi = O.to_conc(mech, st.Y[:, i], st.T[i], st.P[i])
        J, rc = O.jac_conc(mech, st.P[i], phi)
        assert rc == 0
        Jp = J[np.ix_(var, var)]
        assert np.all(Jp[~pat] == 0.0)


def test_unsupported_and_invalid_mechanisms():
    mech = synth.make_mechanism("h2")
    bad = synth.make_mechanism("h2")
    tb = int(np.where(bad.rtype != 0)[0][0])
    bad.eff = bad.eff.copy()
    bad.eff[tb, -1] = 0.7          # a bath gas with a non-default efficiency
    with pytest.raises(kin.KinError) as e:
        kin.conc_analyse(bad)
    assert e.value.code == kin.KIN_ERR_UNSUPPORTED
    bad = synth.make_mechanism("h2")
    bad.reac = bad.reac.copy()
    bad.reac[0, 0] = mech.ns - 1   # the bath gas reacting
    with pytest.raises(kin.KinError) as e:
        kin.conc_analyse(bad)
    assert e.value.code == kin.KIN_ERR_MECH
