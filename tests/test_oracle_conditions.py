"""Pins for several experimental conditions in the oracle (paper Eq. 1d / 2e:
per-condition state profiles and initial conditions, shared theta; Eq. 3:
condition inputs lifted into the right-hand side)."""
import dataclasses

import numpy as np

from paper_2607_12201_gb300 import workloads as W
from oracle import ipm
from oracle.init import forward_sweep
from oracle.nlp import Problem


def _as_conditions(inst, copies):
    """The same single-condition instance stated as `copies` identical conditions."""
    M = inst.M
    return dataclasses.replace(
        inst, cond_x0=np.tile(inst.x0, (copies, 1)), cond_scale=np.ones((copies, inst.r)),
        obs_t=np.tile(inst.obs_t, copies), obs_s=np.tile(inst.obs_s, copies),
        obs_y=np.tile(inst.obs_y, copies), obs_sigma=np.tile(inst.obs_sigma, copies),
        obs_cond=np.repeat(np.arange(copies, dtype=np.int32), M))


def test_one_condition_is_the_plain_problem():
    inst = W.small_network(n=3, r=5, N=6, seed=8)
    one = _as_conditions(inst, 1)
    a, b = Problem(inst), Problem(one)
    rng = np.random.default_rng(2)
    x = rng.uniform(0.2, 1.2, a.n_x)
    lam = rng.standard_normal(a.n_c)
    ea, eb = a.evaluate(x, lam), b.evaluate(x, lam)
    assert ea["phi"] == eb["phi"]
    assert np.array_equal(ea["c"], eb["c"]) and np.array_equal(ea["grad"], eb["grad"])
    assert (ea["J"] != eb["J"]).nnz == 0 and (ea["W"] != eb["W"]).nnz == 0


def test_identical_conditions_double_the_objective_and_keep_the_optimum():
    """Two identical conditions: every constraint block repeats, Phi doubles at
    the repeated point, and the single condition's optimum, repeated, is a KKT
    point of the doubled problem (multipliers repeated, bound duals doubled)."""
    inst = W.config1().with_mesh(10)
    two = _as_conditions(inst, 2)
    p1, p2 = Problem(inst), Problem(two)
    rng = np.random.default_rng(4)
    x1 = rng.uniform(0.2, 1.2, p1.n_x)
    z1, th = p1.split(x1)
    x2 = np.concatenate([np.concatenate([z1, z1]).reshape(-1), th])
    assert np.isclose(p2.objective(x2)[0], 2 * p1.objective(x1)[0], rtol=1e-14)
    c1, c2 = p1.constraints(x1), p2.constraints(x2)
    assert np.array_equal(c2, np.concatenate([c1, c1]))
    opt = ipm.Options(tol=1e-9)
    r1 = ipm.solve(inst, opt=opt)
    assert r1.status == ipm.SUCCESS
    z, th = p1.split(r1.x)
    x2 = np.concatenate([np.concatenate([z, z]).reshape(-1), th])
    lam2 = np.concatenate([r1.lam, r1.lam])
    e1 = ipm.optimality_error(p1, p1.evaluate(r1.x, r1.lam), r1.x, r1.lam, r1.zl, r1.zu, 0.0, opt)
    e2 = ipm.optimality_error(p2, p2.evaluate(x2, lam2), x2, lam2, 2 * r1.zl, 2 * r1.zu, 0.0, opt)
    assert e1 <= 1e-9 and e2 <= 3 * e1 + 1e-12


def test_conditions_couple_only_through_theta():
    """No constraint of one condition involves another condition's states, and
    each condition's first element starts from that condition's x0."""
    inst = W.multi_condition(n=4, r=8, Nc=3, N=5, M=10, seed=31)
    prob = Problem(inst)
    J = prob.jacobian(np.random.default_rng(1).uniform(0.2, 1.0, prob.n_x)).tocoo()
    per = prob.Nch * (prob.K + 1) * prob.n
    for r, c in zip(J.row, J.col):
        if c < prob.nz:
            assert r // per == c // per
    z, fails = forward_sweep(prob, inst.theta_true)
    assert fails == 0
    for c in range(inst.Nc):
        assert np.array_equal(z[c * prob.Nch, 0], inst.cond_x0[c])
    x = np.concatenate([z.reshape(-1), inst.theta_true])
    assert np.max(np.abs(prob.constraints(x))) <= 1e-10


def test_condition_inputs_scale_the_rate_constants():
    """Scaling every rate constant of a condition by u is the same as
    multiplying its right-hand side by u (mass action is linear in k)."""
    inst = W.multi_condition(n=4, r=8, Nc=2, N=4, M=10, seed=32)
    u = 3.0
    scaled = dataclasses.replace(inst, cond_scale=np.vstack([inst.cond_scale[0],
                                                             u * np.ones(inst.r)]))
    base = dataclasses.replace(inst, cond_scale=np.ones((2, inst.r)))
    pb, ps = Problem(base), Problem(scaled)
    rng = np.random.default_rng(5)
    zn = rng.uniform(0.1, 1.0, (3, inst.n))
    th = inst.theta_true
    assert np.allclose(ps.rhs(zn, th, ps.escale[ps.Nch]), u * pb.rhs(zn, th, pb.escale[pb.Nch]),
                       rtol=1e-14, atol=0)


def test_multi_condition_derivatives_match_central_differences():
    inst = W.multi_condition(n=3, r=6, Nc=2, N=3, M=8, seed=33)
    prob = Problem(inst)
    rng = np.random.default_rng(6)
    x = rng.uniform(0.2, 1.0, prob.n_x)
    x[prob.nz:] = rng.uniform(-0.5, 0.5, prob.p)
    lam = rng.standard_normal(prob.n_c)
    ev = prob.evaluate(x, lam, obj_factor=0.7)
    J, Wh = ev["J"].toarray(), ev["W"].toarray()
    eps = 1e-6
    Jfd, Wfd = np.zeros_like(J), np.zeros_like(Wh)

    def lag_grad(xx):
        e = prob.evaluate(xx, lam, obj_factor=0.7)
        return e["grad"] + e["J"].T @ lam

    for a in range(prob.n_x):
        xp, xm = x.copy(), x.copy()
        xp[a] += eps
        xm[a] -= eps
        Jfd[:, a] = (prob.constraints(xp) - prob.constraints(xm)) / (2 * eps)
        Wfd[:, a] = (lag_grad(xp) - lag_grad(xm)) / (2 * eps)
    assert np.max(np.abs(J - Jfd)) <= 1e-7 * max(1.0, np.max(np.abs(J)))
    assert np.max(np.abs(Wh - Wfd)) <= 1e-6 * max(1.0, np.max(np.abs(Wh)))
