"""Pins for the oracle's mesh refinement (defect, interpolation, warm start,
refine-and-resolve loop; paper Section "Static collocation mesh limitations")."""
import numpy as np
import pytest

from paper_2607_12201_gb300 import workloads as W
from oracle import ipm, refine
from oracle.init import forward_sweep
from oracle.nlp import Problem


def test_basis_derivative_matches_the_differentiation_matrix():
    """l_j'(tau_k) are the entries D[k][j] of the collocation equations (Eq. 3)."""
    prob = Problem(W.config1())
    tau = prob.tab.tau
    for k, t in enumerate(tau):
        assert np.allclose(refine.basis_derivative(tau, t), prob.tab.D[k], rtol=0, atol=1e-12)


def test_residual_at_the_collocation_points_is_the_collocation_constraint():
    """At tau_1..tau_K the residual of the defect formula is |c_ik| (Eq. 3), at
    any x: same sign convention, same factor h."""
    inst = W.small_network(n=3, r=5, N=6, seed=8)
    prob = Problem(inst)
    rng = np.random.default_rng(3)
    x = rng.uniform(0.2, 1.2, prob.n_x)
    r = refine.residual_at(prob, x, prob.tab.tau[1:])
    c = prob.constraints(x).reshape(prob.N, prob.K + 1, prob.n)[:, 1:, :]
    assert np.max(np.abs(r - np.abs(c))) <= 1e-13 * max(1.0, np.max(np.abs(c)))


def test_interpolation_is_exact_for_cubic_profiles():
    """States that are one cubic polynomial in t on the whole horizon are
    reproduced exactly at the finer mesh's points (K = 3 Lagrange basis)."""
    inst = W.small_network(n=2, r=3, N=5, seed=21)
    coarse, fine = Problem(inst), Problem(inst.with_mesh(13))
    cubic = lambda t, s: 0.3 + (s + 1) * t - 0.2 * t ** 2 + 0.05 * (s + 2) * t ** 3

    def states(prob):
        z = np.zeros((prob.N, prob.K + 1, prob.n))
        for i in range(prob.N):
            for j in range(prob.K + 1):
                for s in range(prob.n):
                    z[i, j, s] = cubic((i + prob.tab.tau[j]) * prob.h, s)
        return np.concatenate([z.reshape(-1), inst.theta0])

    xf = refine.interpolate(coarse, states(coarse), fine)
    assert np.max(np.abs(xf - states(fine))) <= 1e-12


def test_defect_of_the_collocation_solution_falls_at_order_k_plus_one():
    """Radau collocation with K = 3 on the linear cascade: the residual of the
    collocation polynomial between its points is O(h^K), the defect (h times
    it) O(h^(K+1)) = O(h^4): halving h divides it by about 16."""
    inst = W.config1()
    d = []
    for N in (20, 40, 80):
        prob = Problem(inst.with_mesh(N))
        z, fails = forward_sweep(prob, inst.theta_true)
        assert fails == 0
        d.append(refine.defect(prob, np.concatenate([z.reshape(-1), inst.theta_true]))[1])
    for a, b in zip(d, d[1:]):
        assert 12.0 < a / b < 20.0, d


def test_warm_start_from_the_solution_ends_at_the_same_optimum():
    inst = W.config1()
    first = ipm.solve(inst, opt=ipm.Options(tol=1e-10))
    again = ipm.solve(inst, opt=ipm.Options(tol=1e-10), x_start=first.x)
    assert again.status == ipm.SUCCESS
    assert np.max(np.abs(again.x[-2:] - first.x[-2:])) <= 1e-9


def test_refinement_loop_reaches_the_fine_mesh_optimum():
    """Refining N = 5 -> 10 -> 20 from the interpolated solutions ends at the
    optimum the IPM reaches on N = 20 from the forward sweep."""
    inst = W.config1().with_mesh(5)
    opt = ipm.Options(tol=1e-10)
    out = refine.refine_solve(inst, inst.theta0, opt, defect_tol=1e-12, max_levels=2)
    assert out.levels == 2 and out.inst.N == 20
    assert out.result.status == ipm.SUCCESS
    direct = ipm.solve(inst.with_mesh(20), opt=opt)
    assert np.max(np.abs(out.result.x[-2:] - direct.x[-2:])) <= 1e-8
    # a tolerance above the coarse defect stops at once
    stay = refine.refine_solve(inst, inst.theta0, opt, defect_tol=1e3, max_levels=2)
    assert stay.levels == 0
