"""Pins for the oracle's Gauss-Legendre collocation option (the paper's own node
choice, Eq. 2b-2d / Eq. 3; the GPU path implements Radau IIA, K = 3).

With Gauss-Legendre roots the interior nodes exclude tau = 1, so the state
carried into the next element (Eq. 2c) is the extrapolated end value
``sum_j b_j z_ij`` with ``b_j = l_j(1)``.  Pins:

* the nodes against their closed forms (K = 2, 3, 4) and Gauss quadrature's
  exactness for polynomials of degree <= 2K - 1;
* ``b`` and ``D`` against polynomial exactness;
* for the linear cascade z' = A z, K-stage Gauss collocation advances an
  element by the (K, K) diagonal Pade approximant of exp(hA) (the stability
  function of the K-stage Gauss method), so the sweep's end values are fixed
  in closed form, and their error against exp(At) x0 falls as h^(2K);
* the constraints vanish at the sweep's point and the Jacobian (including the
  new continuity rows) matches central differences."""
import dataclasses
import math

import numpy as np
import pytest
import scipy.linalg as sla

from paper_2607_12201_gb300 import workloads as W
from oracle.init import forward_sweep
from oracle.nlp import Problem
from oracle.radau import Tables

CLOSED = {
    2: [0.5 - math.sqrt(3) / 6, 0.5 + math.sqrt(3) / 6],
    3: [0.5 - math.sqrt(15) / 10, 0.5, 0.5 + math.sqrt(15) / 10],
    4: sorted(0.5 + sg * 0.5 * math.sqrt((3 + sg2 * 2 * math.sqrt(6 / 5)) / 7)
              for sg in (-1, 1) for sg2 in (-1, 1)),
}


@pytest.mark.parametrize("K", [2, 3, 4])
def test_gauss_nodes_closed_form(K):
    tau = Tables(K, "gauss").tau
    assert tau[0] == 0.0
    np.testing.assert_allclose(tau[1:], CLOSED[K], rtol=0, atol=1e-15)


@pytest.mark.parametrize("K", [2, 3, 4, 5])
def test_gauss_quadrature_exact_to_degree_2K_minus_1(K):
    tau = Tables(K, "gauss").tau[1:]
    V = np.vander(tau, K, increasing=True).T               # moments m < K fix the weights
    w = np.linalg.solve(V, 1.0 / np.arange(1, K + 1))
    for m in range(2 * K):
        assert abs(w @ tau ** m - 1.0 / (m + 1)) < 1e-14, m
    assert abs(w @ tau ** (2 * K) - 1.0 / (2 * K + 1)) > 1e-8


@pytest.mark.parametrize("K", [3, 4])
def test_end_weights_and_diff_matrix_exact_for_polynomials(K):
    t = Tables(K, "gauss")
    for m in range(K + 1):
        assert abs(t.b @ t.tau ** m - 1.0) < 1e-13, m          # extrapolation to tau = 1
        dm = m * t.tau ** (m - 1) if m > 0 else np.zeros_like(t.tau)
        np.testing.assert_allclose(t.D @ t.tau ** m, dm, rtol=0, atol=1e-12)
    assert abs(t.b @ t.tau ** (K + 1) - 1.0) > 1e-6
    np.testing.assert_array_equal(Tables(3, "radau").b, [0.0, 0.0, 0.0, 1.0])


def pade_diag(M, K):
    c = [math.factorial(2 * K - j) * math.factorial(K) /
         (math.factorial(2 * K) * math.factorial(j) * math.factorial(K - j)) for j in range(K + 1)]
    I = np.eye(M.shape[0])
    P = sum(cj * np.linalg.matrix_power(M, j) for j, cj in enumerate(c))
    Q = sum(cj * np.linalg.matrix_power(-M, j) for j, cj in enumerate(c))
    return np.linalg.solve(Q, P)


def gauss_cascade(N, K=4):
    return dataclasses.replace(W.linear_cascade(N=N, noise=False), K=K, scheme="gauss")


@pytest.mark.parametrize("N", [4, 25])
def test_gauss_sweep_matches_diagonal_pade(N):
    inst = gauss_cascade(N)
    prob = Problem(inst)
    th = np.array([0.7, 0.3])
    z, fails = forward_sweep(prob, th)
    assert fails == 0
    R = pade_diag(prob.h * np.array([[-th[0], 0.0], [th[0], -th[1]]]), 4)
    zz = inst.x0.copy()
    for i in range(N):
        np.testing.assert_allclose(z[i, 0], zz, rtol=0, atol=1e-14)
        zz = R @ zz
        np.testing.assert_allclose(prob.tab.b @ z[i], zz, rtol=0, atol=5e-14)


def test_gauss_endpoint_order_h8():
    th = np.array([0.7, 0.3])
    A = np.array([[-th[0], 0.0], [th[0], -th[1]]])
    exact = sla.expm(A * 10.0) @ np.array([1.0, 0.0])
    errs = []
    for N in (4, 8, 16):
        prob = Problem(gauss_cascade(N))
        z, _ = forward_sweep(prob, th)
        errs.append(np.max(np.abs(prob.tab.b @ z[-1] - exact)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    for r in rates:
        assert 7.3 < r < 8.7, (errs, rates)


def test_gauss_constraints_vanish_and_jacobian_matches_differences():
    inst = dataclasses.replace(W.small_network(n=3, r=4, N=3, seed=7), K=4, scheme="gauss")
    prob = Problem(inst)
    z, fails = forward_sweep(prob, inst.theta_true)
    assert fails == 0
    x = np.concatenate([z.reshape(-1), inst.theta_true])
    c = prob.constraints(x)
    assert np.max(np.abs(c)) < 1e-12
    # continuity rows carry the extrapolated end value of the previous element
    cz = c.reshape(prob.N, 5, prob.n)
    assert np.max(np.abs(cz[1:, 0])) < 1e-14
    rng = np.random.default_rng(3)
    xp = x * (1.0 + 0.05 * rng.standard_normal(x.size))
    J = prob.jacobian(xp).toarray()
    Jfd = np.zeros_like(J)
    eps = 1e-6
    for a in range(x.size):
        e = np.zeros(x.size); e[a] = eps * max(1.0, abs(xp[a]))
        Jfd[:, a] = (prob.constraints(xp + e) - prob.constraints(xp - e)) / (2 * e[a])
    assert np.max(np.abs(J - Jfd)) <= 1e-7 * max(1.0, np.max(np.abs(J)))


def test_gauss_ipm_agrees_with_radau_estimate():
    # two discretisations of the same estimation problem: the estimates differ
    # by the discretisation error only (Radau K = 3: h^5, Gauss K = 4: h^8)
    from oracle import ipm as oipm
    base = W.linear_cascade(N=20)
    rr = oipm.solve(base)
    rg = oipm.solve(dataclasses.replace(base, K=4, scheme="gauss"))
    assert rr.status == 0 and rg.status == 0
    tr, tg = rr.x[-base.p:], rg.x[-base.p:]
    assert np.max(np.abs(tg - tr) / np.abs(tr)) < 1e-5
    assert np.max(np.abs(tg - tr)) > 0.0
