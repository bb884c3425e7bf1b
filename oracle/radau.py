"""Collocation tables (oracle; test infrastructure only).

Paper, Eq. 2b / Eq. 3: the collocation constraint of element i, node k is
``sum_j a_j(tau_k) z_ij = h_i f(z_ik, theta)`` with ``a_j(tau_k)`` the tau
derivative of the j-th Lagrange basis polynomial of degree K on the K+1
interpolation points ``tau_0 = 0 < tau_1 < ... < tau_K``, and the
continuity constraint of Eq. 2c carries the state at the element's end,
``sum_j b_j z_ij`` with ``b_j = l_j(1)``, into the next element.  The paper
uses Gauss-Legendre roots; the GPU path uses right Radau (Radau IIA) roots,
for which ``tau_K = 1`` and ``b_j = delta_jK``.  Both are tabulated here.

* Radau: ``tau[1..K]`` are the roots of ``P_K(x) - P_{K-1}(x)`` mapped from
  [-1, 1] to [0, 1] (P = Legendre polynomials), found by numpy's Legendre
  root finder and polished by Newton iterations on the three-term
  recurrence.
* Gauss-Legendre: ``tau[1..K]`` are the roots of ``P_K``, mapped and
  polished the same way.
* ``b_j = l_j(1)`` (exactly ``delta_jK`` for Radau).
* ``D[k][j] = l_j'(tau_k)``: derivative of the Lagrange basis, from the
  barycentric formula ``D[k][j] = (w_j / w_k) / (tau_k - tau_j)``,
  ``D[k][k] = -sum_{j != k} D[k][j]``.
* ``basis(t)[j] = l_j(t)``: product formula.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg


def _legendre_and_derivative(K: int, x: float):
    """P_K(x) and P'_K(x) by the Bonnet recurrence."""
    p_prev, p = 1.0, x
    if K == 0:
        return 1.0, 0.0
    for m in range(1, K):
        p_prev, p = p, ((2 * m + 1) * x * p - m * p_prev) / (m + 1)
    dp = K * (x * p - p_prev) / (x * x - 1.0) if abs(x) != 1.0 else K * (K + 1) / 2 * x ** (K + 1)
    return p, dp


def radau_nodes(K: int) -> np.ndarray:
    """Interpolation points [0, tau_1, ..., tau_K] with tau_K = 1."""
    coef = np.zeros(K + 1)
    coef[K] = 1.0
    coef[K - 1] = -1.0
    roots = np.sort(np.real(npleg.legroots(coef)))
    polished = []
    for x in roots:
        if abs(x - 1.0) < 1e-12:
            polished.append(1.0)
            continue
        for _ in range(20):
            pk, dpk = _legendre_and_derivative(K, x)
            pk1, dpk1 = _legendre_and_derivative(K - 1, x)
            step = (pk - pk1) / (dpk - dpk1)
            x -= step
            if abs(step) < 1e-17:
                break
        polished.append(x)
    tau = np.concatenate([[0.0], (np.array(polished) + 1.0) / 2.0])
    tau[-1] = 1.0
    return tau


def gauss_nodes(K: int) -> np.ndarray:
    """Interpolation points [0, tau_1, ..., tau_K], tau_k the Gauss-Legendre roots."""
    coef = np.zeros(K + 1)
    coef[K] = 1.0
    roots = np.sort(np.real(npleg.legroots(coef)))
    polished = []
    for x in roots:
        for _ in range(20):
            pk, dpk = _legendre_and_derivative(K, x)
            step = pk / dpk
            x -= step
            if abs(step) < 1e-17:
                break
        polished.append(x)
    return np.concatenate([[0.0], (np.array(polished) + 1.0) / 2.0])


def barycentric_weights(tau: np.ndarray) -> np.ndarray:
    w = np.ones_like(tau)
    for j in range(len(tau)):
        for m in range(len(tau)):
            if m != j:
                w[j] /= (tau[j] - tau[m])
    return w


def diff_matrix(tau: np.ndarray) -> np.ndarray:
    """D[k][j] = d l_j / d tau evaluated at tau_k."""
    w = barycentric_weights(tau)
    npts = len(tau)
    D = np.zeros((npts, npts))
    for k in range(npts):
        for j in range(npts):
            if j != k:
                D[k, j] = (w[j] / w[k]) / (tau[k] - tau[j])
        D[k, k] = -np.sum(D[k, :])
    return D


def basis(tau: np.ndarray, t: float) -> np.ndarray:
    """l_j(t) for j = 0..K."""
    out = np.ones(len(tau))
    for j in range(len(tau)):
        for m in range(len(tau)):
            if m != j:
                out[j] *= (t - tau[m]) / (tau[j] - tau[m])
    return out


class Tables:
    def __init__(self, K: int = 3, scheme: str = "radau"):
        if scheme not in ("radau", "gauss"):
            raise ValueError(f"unknown collocation scheme {scheme!r}")
        self.K = K
        self.scheme = scheme
        self.tau = radau_nodes(K) if scheme == "radau" else gauss_nodes(K)
        self.D = diff_matrix(self.tau)
        self.b = basis(self.tau, 1.0)      # continuity weights, Eq. 2c
