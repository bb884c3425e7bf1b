"""Pins for the oracle's collocation tables (Eq. 3: Lagrange basis on Radau points)."""
import math

import numpy as np
import pytest

from oracle.radau import Tables, basis, diff_matrix, radau_nodes


def test_radau_k3_nodes_closed_form():
    # Radau IIA, K = 3: tau = (4 -+ sqrt 6)/10 and 1 (Hairer & Wanner, Table IV.5.5)
    tau = radau_nodes(3)
    s6 = math.sqrt(6.0)
    np.testing.assert_allclose(tau, [0.0, (4 - s6) / 10, (4 + s6) / 10, 1.0], rtol=0, atol=1e-15)


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5])
def test_radau_nodes_are_roots_and_superconvergent_quadrature(K):
    tau = radau_nodes(K)
    assert tau[0] == 0.0 and tau[-1] == 1.0
    assert np.all(np.diff(tau) > 0)
    # Radau quadrature on the K nodes is exact for degree 2K-2: weights b_j = int l_j
    nodes = tau[1:]
    V = np.vander(nodes, K, increasing=True).T          # V[d, j] = nodes_j^d
    b = np.linalg.solve(V, 1.0 / np.arange(1, K + 1))
    for d in range(2 * K - 1):
        assert abs(b @ nodes ** d - 1.0 / (d + 1)) < 1e-13
    # ... and not for degree 2K-1 (K >= 1)
    d = 2 * K - 1
    assert abs(b @ nodes ** d - 1.0 / (d + 1)) > 1e-8


def test_diff_matrix_row_sums_and_polynomial_exactness():
    tau = radau_nodes(3)
    D = diff_matrix(tau)
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-13)
    for deg in range(0, 4):
        vals = tau ** deg
        exact = deg * tau ** (deg - 1) if deg > 0 else np.zeros_like(tau)
        np.testing.assert_allclose(D @ vals, exact, atol=1e-12)
    # a quartic is NOT differentiated exactly by a cubic interpolant
    assert np.max(np.abs(D @ tau ** 4 - 4 * tau ** 3)) > 1e-3


def test_diff_matrix_interior_block_inverts_to_radau_butcher_matrix():
    # The collocation stage equations sum_j D[k][j] z_j = h f_k are the Radau IIA
    # Runge-Kutta method: A = (D[1:,1:])^{-1}, the published Butcher matrix.
    s6 = math.sqrt(6.0)
    A_pub = np.array([
        [(88 - 7 * s6) / 360, (296 - 169 * s6) / 1800, (-2 + 3 * s6) / 225],
        [(296 + 169 * s6) / 1800, (88 + 7 * s6) / 360, (-2 - 3 * s6) / 225],
        [(16 - s6) / 36, (16 + s6) / 36, 1.0 / 9.0]])
    D = Tables(3).D
    np.testing.assert_allclose(np.linalg.inv(D[1:, 1:]), A_pub, atol=1e-14)


def test_basis_cardinal_partition_and_interpolation():
    tau = radau_nodes(3)
    for i, t in enumerate(tau):
        e = np.zeros(4)
        e[i] = 1.0
        np.testing.assert_allclose(basis(tau, t), e, atol=1e-15)
    rng = np.random.default_rng(0)
    coef = rng.standard_normal(4)
    for t in rng.uniform(0, 1, 10):
        assert abs(basis(tau, t).sum() - 1.0) < 1e-14
        assert abs(basis(tau, t) @ np.polyval(coef, tau) - np.polyval(coef, t)) < 1e-13
