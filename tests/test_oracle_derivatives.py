"""Pins for the oracle's first and second derivatives by central differences."""
import numpy as np
import pytest

from paper_2607_12201_gb300 import workloads as W
from oracle.nlp import Problem


def _point(prob, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.2, 1.0, prob.n_x)
    if prob.inst.logscale:
        x[prob.nz:] = rng.uniform(-0.5, 0.5, prob.p)
    else:
        x[prob.nz:] = rng.uniform(0.2, 1.0, prob.p)
    lam = rng.standard_normal(prob.n_c)
    return x, lam


@pytest.mark.parametrize("make", [lambda: W.small_network(n=3, r=5, N=3, seed=11),
                                  lambda: W.small_network(n=4, r=6, N=2, seed=12),
                                  lambda: W.linear_cascade(N=3)])
def test_jacobian_gradient_hessian_by_central_differences(make):
    inst = make()
    prob = Problem(inst)
    x, lam = _point(prob, 1)
    ev = prob.evaluate(x, lam, obj_factor=0.7)
    J, Wh = ev["J"].toarray(), ev["W"].toarray()
    eps = 1e-6
    Jfd = np.zeros_like(J)
    gfd = np.zeros(prob.n_x)
    Wfd = np.zeros_like(Wh)

    def lag_grad(xx):
        e = prob.evaluate(xx, lam, obj_factor=0.7)
        return e["grad"] + e["J"].T @ lam

    for a in range(prob.n_x):
        xp, xm = x.copy(), x.copy()
        xp[a] += eps
        xm[a] -= eps
        Jfd[:, a] = (prob.constraints(xp) - prob.constraints(xm)) / (2 * eps)
        gfd[a] = 0.7 * (prob.objective(xp)[0] - prob.objective(xm)[0]) / (2 * eps)
        Wfd[:, a] = (lag_grad(xp) - lag_grad(xm)) / (2 * eps)
    assert np.max(np.abs(J - Jfd)) <= 1e-7 * max(1.0, np.max(np.abs(J)))
    assert np.max(np.abs(ev["grad"] - gfd)) <= 1e-6 * max(1.0, np.max(np.abs(gfd)))
    assert np.max(np.abs(Wh - Wfd)) <= 1e-6 * max(1.0, np.max(np.abs(Wh)))
    assert np.max(np.abs(Wh - Wh.T)) <= 1e-14 * max(1.0, np.max(np.abs(Wh)))


def test_objective_matches_direct_definition():
    inst = W.small_network(n=3, r=4, N=5, seed=3, M=7)
    prob = Problem(inst)
    x, _ = _point(prob, 2)
    z, _ = prob.split(x)
    phi, _ = prob.objective(x)
    # direct: cubic through (t_ij, z_ij) on the observation's element, evaluated at t_m
    h = inst.T / inst.N
    total = 0.0
    tau = prob.tab.tau
    for m in range(inst.M):
        t = inst.obs_t[m]
        i = min(max(int(np.ceil(t / h - 1e-12)) - 1, 0), inst.N - 1)
        ts = i * h + h * tau
        coef = np.polyfit(ts, z[i, :, inst.obs_s[m]], 3)
        yhat = np.polyval(coef, t)
        total += 0.5 * ((yhat - inst.obs_y[m]) / inst.obs_sigma[m]) ** 2
    assert abs(phi - total) <= 1e-9 * max(1.0, total)


def test_mass_action_rhs_on_hand_written_network():
    # A + B -> C (k0), C -> A (k1), 2B -> nothing... use react/prod slots directly
    inst = W.small_network(n=3, r=3, N=1, seed=5)
    inst.react[:] = [[0, 1], [2, -1], [1, 1]]
    inst.prod[:] = [[2, -1], [0, -1], [-1, -1]]
    prob = Problem(inst)
    th = np.array([0.1, -0.2, 0.3])
    k = 10.0 ** th
    z = np.array([0.5, 0.7, 0.9])
    v = [k[0] * z[0] * z[1], k[1] * z[2], k[2] * z[1] * z[1]]
    f_exp = np.array([-v[0] + v[1], -v[0] - 2 * v[2], v[0] - v[1]])
    np.testing.assert_allclose(prob.rhs(z[None], th)[0], f_exp, rtol=1e-15)


def test_observations_on_element_boundaries_use_the_left_element():
    # Reading of the observation model for times on the mesh: a time on an
    # element boundary belongs to the element on its left (tau = 1, i.e. its end
    # state z_iK), t = 0 to the first element's start state z_10.  At a point
    # that violates continuity the two neighbours disagree, so the choice shows.
    import dataclasses
    base = W.small_network(n=3, r=4, N=4, seed=3, M=5, T=2.0)
    h = base.T / base.N                                   # 0.5, exact in binary
    times = np.array([0.0, h, 2 * h, 3 * h, base.T])
    species = np.array([0, 1, 2, 0, 1], dtype=base.obs_s.dtype)
    y = np.array([0.3, 0.4, 0.5, 0.6, 0.7])
    sig = np.array([0.1, 0.2, 0.1, 0.3, 0.1])
    inst = dataclasses.replace(base, obs_t=times, obs_s=species, obs_y=y, obs_sigma=sig)
    prob = Problem(inst)
    x, _ = _point(prob, 4)
    z, _ = prob.split(x)
    K = prob.K
    yhat = [z[0, 0, 0], z[0, K, 1], z[1, K, 2], z[2, K, 0], z[3, K, 1]]
    assert abs(z[0, K, 1] - z[1, 0, 1]) > 1e-3              # the neighbours disagree
    expected = 0.5 * sum(((yh - yy) / s) ** 2 for yh, yy, s in zip(yhat, y, sig))
    phi, _ = prob.objective(x)
    assert abs(phi - expected) <= 1e-13 * max(1.0, expected)


@pytest.mark.parametrize("scheme", ["radau3", "gauss4"])
@pytest.mark.parametrize("make", [lambda: W.small_network(n=3, r=5, N=3, seed=11),
                                  lambda: W.small_network(n=4, r=6, N=2, seed=12),
                                  lambda: W.linear_cascade(N=3)])
def test_derivatives_by_fourth_order_differences(make, scheme):
    # five-point stencil (f(x-2e) - 8 f(x-e) + 8 f(x+e) - f(x+2e)) / (12 e), truncation
    # error O(e^4): the constraints are at most quadratic in the states and smooth in
    # theta, so with e = 1e-3 the differences are accurate to ~1e-11 and pin every
    # derivative entry to 1e-9 relative -- a missing term far below the size of the
    # largest entries fails here
    import dataclasses
    inst = make()
    if scheme == "gauss4":
        inst = dataclasses.replace(inst, K=4, scheme="gauss")
    prob = Problem(inst)
    x, lam = _point(prob, 3)
    of = 1.3
    ev = prob.evaluate(x, lam, obj_factor=of)
    J, Wh, g = ev["J"].toarray(), ev["W"].toarray(), ev["grad"]

    def lag_grad(xx):
        e = prob.evaluate(xx, lam, obj_factor=of)
        return e["grad"] + e["J"].T @ lam

    def d5(fun, a, e=1e-3):
        vals = []
        for s in (-2, -1, 1, 2):
            xx = x.copy()
            xx[a] += s * e
            vals.append(fun(xx))
        return (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * e)

    Jfd = np.column_stack([d5(prob.constraints, a) for a in range(prob.n_x)])
    gfd = np.array([of * d5(lambda xx: prob.objective(xx)[0], a) for a in range(prob.n_x)])
    Wfd = np.column_stack([d5(lag_grad, a) for a in range(prob.n_x)])
    assert np.max(np.abs(J - Jfd)) <= 1e-9 * max(1.0, np.max(np.abs(J)))
    assert np.max(np.abs(g - gfd)) <= 1e-9 * max(1.0, np.max(np.abs(g)))
    assert np.max(np.abs(Wh - Wfd)) <= 1e-9 * max(1.0, np.max(np.abs(Wh)))
