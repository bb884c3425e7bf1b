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


# K = 2 Gauss (Hammer-Hollingsworth) Butcher tableau, published in closed form.
_S3 = math.sqrt(3.0)
_C2 = np.array([0.5 - _S3 / 6, 0.5 + _S3 / 6])
_A2 = np.array([[0.25, 0.25 - _S3 / 6], [0.25 + _S3 / 6, 0.25]])
_B2 = np.array([0.5, 0.5])


def _reduced_gauss2(theta, inst):
    """Weighted misfit of the K = 2 Gauss Runge-Kutta discretisation (stage
    equations by Newton per element, end value y0 + h sum_j b_j f(Z_j), model
    output from the quadratic through (0, c_1, c_2))."""
    from test_oracle_ipm import _mass_action, _rate_constants
    k = _rate_constants(theta, inst)
    n, h = inst.n, inst.T / inst.N
    z0 = np.array(inst.x0, dtype=float)
    pts = []
    for _ in range(inst.N):
        Z = np.tile(z0, (2, 1))
        for _ in range(50):
            fj = [_mass_action(Z[l], k, inst) for l in range(2)]
            F = np.array([Z[a] - z0 - h * sum(_A2[a, l] * fj[l][0] for l in range(2)) for a in range(2)])
            Jb = np.block([[(np.eye(n) if a == l else 0.0 * np.eye(n)) - h * _A2[a, l] * fj[l][1]
                            for l in range(2)] for a in range(2)])
            d = np.linalg.solve(Jb, F.reshape(-1)).reshape(2, n)
            Z = Z - d
            if np.max(np.abs(d)) < 1e-15 * max(1.0, np.max(np.abs(Z))):
                break
        pts.append((z0.copy(), Z.copy()))
        fj = [_mass_action(Z[l], k, inst)[0] for l in range(2)]
        z0 = z0 + h * (_B2[0] * fj[0] + _B2[1] * fj[1])
    res = []
    for m in range(inst.M):
        t = inst.obs_t[m]
        i = min(max(int(math.ceil(t * inst.N / inst.T)) - 1, 0), inst.N - 1)
        zs, Z = pts[i]
        s = inst.obs_s[m]
        vals = np.array([zs[s], Z[0, s], Z[1, s]])
        yhat = np.polyval(np.polyfit(h * np.array([0.0, _C2[0], _C2[1]]), vals, 2), t - i * h)
        res.append((yhat - inst.obs_y[m]) / inst.obs_sigma[m])
    return np.array(res)


def test_gauss_k2_ipm_matches_reduced_space_runge_kutta():
    from scipy.optimize import least_squares
    from oracle import ipm as oipm
    base = W.random_network(3, 4, n_obs=3, M=30, T=5.0, N=12, seed=7, theta0_spread=0.1)
    inst = dataclasses.replace(base, K=2, scheme="gauss")
    ref = least_squares(_reduced_gauss2, inst.theta0, args=(inst,), xtol=1e-15, ftol=1e-15,
                        gtol=1e-15, method="lm")
    res = oipm.solve(inst, opt=oipm.Options(tol=1e-10))
    assert res.status == oipm.SUCCESS
    th = res.x[-inst.p:]
    assert np.max(np.abs(th - ref.x) / np.abs(ref.x)) < 1e-6, (th, ref.x)
    assert abs(res.phi - 0.5 * np.sum(ref.fun ** 2)) < 1e-10 * res.phi
