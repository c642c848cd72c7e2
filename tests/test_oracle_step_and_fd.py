"""Pins of two oracle functions that every integration passes through.

* orc_initial_step, the starting-step heuristic of Hairer, Norsett & Wanner
  Vol. I Sec. II.4 (the first internal step of the Radau IIA integrator of
  Sec. 2.1): worked by hand on linear problems, each case chosen so that a
  different branch of the rule decides (tests/golden/starting_step_cases.txt).
* orc_fd_jacobian, the one-sided difference-quotient Jacobian with CVODE's
  increment rule (Sec. 2.1, Sec. 3.4): on quadratic right-hand sides whose
  increments and quotients are binary numbers, so the expected entries,
  including the forward quotient's truncation term, are exact
  (tests/golden/fd_jacobian_cases.txt).
"""
import os

import numpy as np
import pytest

from conftest import ROOT
from oracle import oracle as O


def _golden(name):
    return os.path.join(ROOT, "tests", "golden", name)


def _starting_cases():
    out = []
    for line in open(_golden("starting_step_cases.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, y0, lam, rtol, atol, span, h = (x.strip() for x in line.split(";"))
        out.append((name, eval(y0), eval(lam), float(rtol), float(atol), float(span), eval(h)))
    return out


@pytest.mark.parametrize("case", _starting_cases(), ids=lambda c: c[0])
def test_starting_step_worked_cases(case):
    name, y0, lam, rtol, atol, span, expected = case
    lam = np.array(lam)
    h, nf = O.initial_step(lambda t, y: lam * y, y0, 0.0, span, rtol, atol)
    assert nf == 1                       # one extra right-hand side: f(y + h0 f0)
    assert abs(h - expected) <= 1e-15 * expected, (name, h, expected)


def test_starting_step_failed_trial_evaluation():
    """A failing f(y + h0 f0) falls back to 0.01 h0 (the integrator's reading
    of a non-finite trial value): lam = -100, sc = 1 gives h0 = 1e-4."""
    def f(t, y):
        return -100.0 * y if t == 0.0 else np.full_like(y, np.nan)
    h, _ = O.initial_step(f, [1.0], 0.0, 1.0, 0.5, 0.5)
    assert abs(h - 0.01 * 1e-4) <= 1e-15 * 1e-6


def _fd_cases():
    out = {}
    for line in open(_golden("fd_jacobian_cases.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        case, entry = (x.strip() for x in line.split(";"))
        key, val = (x.strip() for x in entry.split("="))
        out.setdefault(case, []).append((int(key[1]), int(key[2]), eval(val)))
    return out


FD_PROBLEMS = {
    "relative": (lambda t, y: np.array([y[0] ** 2, y[0] * y[1], y[1] ** 2]),
                 [2.0 ** 20, 2.0 ** 10, 5.0], 1e-30, [1.0, 1.0, 1.0]),
    "floor": (lambda t, y: np.array([y[1] ** 2, y[2] ** 2, 2.0 * y[0], 2.0]),
              [0.0, 0.0, 0.0, 0.0], 2.0 ** -10, [1.0, 1.0, 4.0, 1.0]),
}


@pytest.mark.parametrize("case", sorted(FD_PROBLEMS))
def test_fd_jacobian_exact_on_quadratics(case):
    f, y, h, scal = FD_PROBLEMS[case]
    J, rc = O.fd_jacobian(f, y, h, scal)
    assert rc == 0
    entries = _fd_cases()[case]
    assert len(entries) >= 5
    for i, j, v in entries:
        assert J[i, j] == v, (case, i, j, J[i, j], v)


def test_chemistry_fd_jacobian_is_the_generic_rule(h2_mech):
    """orc_jac_fd is orc_fd_jacobian applied to the chemistry's right-hand side."""
    from paper_1607_03884_gb300 import synth
    om = O.OracleMech(h2_mech)
    st = synth.make_states(h2_mech, 3, seed=5)
    y = O.state_vector(st)
    for i in range(3):
        P = st.P[i]
        f0, _ = O.rhs(om, P, y[:, i])
        scal = 1e-9 + 1e-5 * np.abs(y[:, i])
        Ja, _ = O.jac_fd(om, P, y[:, i], f0, 1e-8, scal)
        Jb, _ = O.fd_jacobian(lambda t, v: O.rhs(om, P, v)[0], y[:, i], 1e-8, scal)
        np.testing.assert_array_equal(Ja, Jb)
