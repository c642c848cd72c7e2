"""Pins of the oracle's dense LU (real and complex) against known solutions,
numpy's LAPACK solve, the pivoting convention and singular detection."""
import numpy as np
import pytest

from oracle import oracle as O


@pytest.mark.parametrize("n", [1, 2, 13, 53])
def test_real_lu_solves_known_system(n):
    rng = np.random.default_rng(n)
    A = rng.normal(size=(n, n)) + n * np.eye(n) * rng.choice([-1, 1], size=n)
    x = rng.normal(size=n)
    lu, ip, rc = O.lu_real(A)
    assert rc == 0
    got = O.lu_solve_real(lu, ip, A @ x)
    np.testing.assert_allclose(got, x, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(got, np.linalg.solve(A, A @ x), rtol=1e-11, atol=1e-12)
    # P A = L U reconstruction
    L = np.tril(lu, -1) + np.eye(n)
    U = np.triu(lu)
    PA = A.copy()
    for k in range(n):
        PA[[k, ip[k]]] = PA[[ip[k], k]]
    np.testing.assert_allclose(L @ U, PA, rtol=1e-12, atol=1e-12 * np.abs(A).max())


@pytest.mark.parametrize("n", [1, 3, 13, 53])
def test_complex_lu_solves_known_system(n):
    rng = np.random.default_rng(100 + n)
    A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)) + 2 * n * np.eye(n)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    lu, ip, rc = O.lu_cplx(A)
    assert rc == 0
    got = O.lu_solve_cplx(lu, ip, A @ x)
    np.testing.assert_allclose(got, x, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(got, np.linalg.solve(A, A @ x), rtol=1e-11, atol=1e-12)


def test_pivot_is_first_largest():
    A = np.array([[1.0, 2.0, 0.0], [-3.0, 1.0, 0.0], [3.0, 0.0, 1.0]])
    lu, ip, rc = O.lu_real(A)
    assert ip[0] == 1          # |-3| ties |3|: the first index wins
    Ac = np.array([[1 + 1j, 0], [2 - 0.0j, 1]])    # |Re|+|Im|: 2 == 2, first wins
    lu, ip, rc = O.lu_cplx(Ac)
    assert ip[0] == 0


def test_singular_matrix_reports_column():
    A = np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [0.0, 0.0, 0.0]])
    _, _, rc = O.lu_real(A)
    assert rc == 2
    _, _, rc = O.lu_cplx(np.zeros((2, 2), dtype=complex))
    assert rc == 1
