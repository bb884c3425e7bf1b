"""Pins for the oracle's collocation discretisation (Eq. 2b-2d, Eq. 3).

For a linear ODE z' = A z, Radau IIA collocation with K = 3 maps the state at
the start of an element to its end by the (2, 3) Pade approximant of exp:
``z_iK = R(hA) z_i0``, ``R(s) = (1 + 2s/5 + s^2/20) / (1 - 3s/5 + 3s^2/20 - s^3/60)``.
The endpoint error against ``exp(At) x0`` is O(h^(2K-1)) = O(h^5).
"""
import numpy as np
import pytest
import scipy.linalg as sla

from paper_2607_12201_gb300 import workloads as W
from oracle.init import forward_sweep
from oracle.nlp import Problem


def pade23(M):
    I = np.eye(M.shape[0])
    P = I + 2 * M / 5 + M @ M / 20
    Q = I - 3 * M / 5 + 3 * M @ M / 20 - M @ M @ M / 60
    return np.linalg.solve(Q, P)


def cascade_matrix(t1, t2):
    return np.array([[-t1, 0.0], [t1, -t2]])


@pytest.mark.parametrize("N", [5, 50])
def test_forward_sweep_matches_pade_closed_form(N):
    inst = W.linear_cascade(N=N, noise=False)
    prob = Problem(inst)
    th = np.array([0.7, 0.3])
    z, fails = forward_sweep(prob, th)
    assert fails == 0
    R = pade23(prob.h * cascade_matrix(*th))
    zz = inst.x0.copy()
    for i in range(N):
        np.testing.assert_allclose(z[i, 0], zz, rtol=0, atol=1e-14)
        zz = R @ zz
        np.testing.assert_allclose(z[i, 3], zz, rtol=0, atol=2e-14)


def test_pade_is_the_radau_stability_function():
    # scalar check of R against exp for small s: R(s) - e^s = O(s^6)
    for s in [-0.3, -2.0, -50.0]:
        r = pade23(np.array([[s]]))[0, 0]
        inst = W.linear_cascade(N=1, T=1.0, noise=False)
        prob = Problem(inst)
        # one element, scalar decay through species 0: x1' = -t1 x1 with t1 = -s
        z, _ = forward_sweep(prob, np.array([-s, 1.0]))
        assert abs(z[0, 3, 0] - r) < 1e-13 * max(1.0, abs(r))


def test_endpoint_order_h5():
    th = np.array([0.7, 0.3])
    A = cascade_matrix(*th)
    exact = sla.expm(A * 10.0) @ np.array([1.0, 0.0])
    errs = []
    Ns = [25, 50, 100]
    for N in Ns:
        prob = Problem(W.linear_cascade(N=N, noise=False))
        z, _ = forward_sweep(prob, th)
        errs.append(np.max(np.abs(z[-1, 3] - exact)))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    for r in rates:
        assert 4.6 < r < 5.4, (errs, rates)


def test_collocation_residual_zero_at_sweep_and_continuity():
    inst = W.small_network(n=3, r=4, N=6)
    prob = Problem(inst)
    z, fails = forward_sweep(prob, inst.theta_true)
    assert fails == 0
    x = np.concatenate([z.reshape(-1), inst.theta_true])
    c = prob.constraints(x)
    assert np.max(np.abs(c)) < 1e-12
