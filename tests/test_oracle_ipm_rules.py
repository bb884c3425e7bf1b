"""Pins for the interior-point rules of the oracle that decide statuses and
iteration counts (Waechter & Biegler 2006, "On the implementation of an
interior-point filter line-search algorithm for large-scale nonlinear
programming", Math. Program. 106): the scaled optimality error, the
acceptable-termination counter, the minimum step alpha_min, the filter /
switching-condition / Armijo acceptance of trial points, the halving sequence
and its failure exit, and the bound-multiplier safeguard.

Expected values are worked out by hand in the comments, not recomputed with
the oracle's formulas.
"""
import math
import types

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2607_12201_gb300 import workloads as W
from oracle import ipm

OPT = ipm.Options()


# ---- scaled optimality error E_mu (Eq. (5)) -----------------------------------------

def _fake_problem():
    """Two states, one parameter theta in [0, 2], two constraints."""
    inst = types.SimpleNamespace(theta_lo=np.array([0.0]), theta_hi=np.array([2.0]))
    return types.SimpleNamespace(inst=inst, nz=2, p=1, n_c=2, n_x=3)


def _fake_point(c):
    # x = (., ., theta = 0.5): slacks s_L = 0.5, s_U = 1.5
    x = np.array([3.0, -1.0, 0.5])
    lam = np.array([1000.0, -1000.0])
    zl, zu = np.array([300.0]), np.array([100.0])
    J = sp.csr_matrix(np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]]))
    grad = np.array([-990.0, 1003.0, 7.0])
    return x, lam, zl, zu, dict(grad=grad, J=J, c=np.asarray(c, dtype=np.float64))


def test_optimality_error_scaling_worked_by_hand():
    """Hand-worked E_mu with s_d != 1 and s_c != 1.

    dual = grad + J^T lam - z_L + z_U = (-990 + 1000, 1003 - 1000, 7 - 300 + 100)
         = (10, 3, -193)                                   -> ||.||_inf = 193
    s_d = max(100, (||lam||_1 + ||z||_1) / (m + 2p)) / 100
        = max(100, (2000 + 400) / (2 + 2)) / 100 = 6     (m + p would give 8)
    s_c = max(100, ||z||_1 / (2p)) / 100 = max(100, 400 / 2) / 100 = 2
                                                       (dividing by p would give 4)
    complementarity: s_L z_L = 0.5 * 300 = 150, s_U z_U = 1.5 * 100 = 150.
    """
    prob = _fake_problem()
    x, lam, zl, zu, ev = _fake_point([0.25, -4.0])
    # mu = 150 cancels the complementarity: E = max(193 / 6, 4, 0)
    assert ipm.optimality_error(prob, ev, x, lam, zl, zu, 150.0, OPT) == pytest.approx(193.0 / 6.0,
                                                                                     rel=1e-15)
    # mu = 0: the complementarity term 150 / 2 = 75 dominates 193 / 6 and 4
    assert ipm.optimality_error(prob, ev, x, lam, zl, zu, 0.0, OPT) == pytest.approx(75.0, rel=1e-15)
    # an infeasibility of 400 dominates everything (it is never scaled)
    x, lam, zl, zu, ev = _fake_point([0.25, -400.0])
    assert ipm.optimality_error(prob, ev, x, lam, zl, zu, 150.0, OPT) == 400.0


def test_optimality_error_unscaled_for_small_multipliers():
    """With ||lam||_1 + ||z||_1 below s_max (m + 2p) and ||z||_1 below s_max 2p both
    scalings are 1: E_0 = max(|dual|_inf, |c|_inf, |s z|_inf)."""
    prob = _fake_problem()
    x = np.array([0.0, 0.0, 0.5])
    lam = np.array([2.0, -1.0])
    zl, zu = np.array([4.0]), np.array([1.0])
    J = sp.csr_matrix(np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]]))
    # dual = (0.5 + 2, 0.25 - 1, 1 - 4 + 1) = (2.5, -0.75, -2)
    ev = dict(grad=np.array([0.5, 0.25, 1.0]), J=J, c=np.array([0.1, 0.2]))
    # complementarity at mu = 0: 0.5 * 4 = 2 and 1.5 * 1 = 1.5
    assert ipm.optimality_error(prob, ev, x, lam, zl, zu, 0.0, OPT) == 2.5
    # at mu = 2 the complementarity terms are |2 - 2| = 0 and |1.5 - 2| = 0.5
    lam2 = np.array([0.0, 0.0])
    ev2 = dict(grad=np.array([0.0, 0.0, 3.0]), J=J, c=np.array([0.1, -0.3]))   # dual = (0, 0, 0)
    assert ipm.optimality_error(prob, ev2, x, lam2, zl, zu, 2.0, OPT) == 0.5


# ---- acceptable termination counter ----------------------------------------------------

def _first_window(errs, thr, width):
    """First index k whose `width` most recent errors (errs[k-width+1..k]) are
    all <= thr, found by scanning windows (no counter)."""
    for k in range(width - 1, len(errs)):
        if all(e <= thr for e in errs[k - width + 1:k + 1]):
            return k
    return None


def test_acceptable_termination_needs_consecutive_iterations():
    """The counter counts consecutive iterates with E_0 <= acceptable_tol and is
    reset by any iterate above it (paper, "Optimization framework
    configurations": acceptable level 1e-4 for 15 iterations; Waechter & Biegler
    2006, Section 3.9).  A reference run that never terminates early gives the
    sequence of E_0; for thresholds where that sequence dips below and back
    above, the solve with acceptable_iter = w must stop exactly at the first
    window of w consecutive iterates below the threshold."""
    inst = W.small_network(n=3, r=5, N=12, seed=8)
    ref = ipm.solve(inst, opt=ipm.Options(tol=1e-12, acceptable_iter=10 ** 6))
    errs = [h["err"] for h in ref.history] + [ref.kkt_error]
    checked = 0
    for thr in sorted(set(errs)):
        for width in (2, 3):
            k = _first_window(errs, thr, width)
            if k is None or k + 1 >= len(errs):
                continue
            below = [e <= thr for e in errs[:k + 1]]
            # only thresholds where the counter must have been reset once
            if not any(below[j] and not below[j + 1] for j in range(k)):
                continue
            res = ipm.solve(inst, opt=ipm.Options(tol=1e-12, acceptable_tol=thr,
                                                  acceptable_iter=width))
            assert res.status == ipm.ACCEPTABLE
            assert res.iterations == k, (thr, width, k, res.iterations)
            checked += 1
            if checked >= 3:
                return
    assert checked > 0, "no non-monotone error sequence to check the reset on"


# ---- minimum step (Eq. (23)) -------------------------------------------------------------

def test_alpha_min_branches_worked_by_hand():
    """gamma_alpha = 0.05, gamma_theta = gamma_phi = 1e-5, delta = 1,
    s_theta = 1.1, s_phi = 2.3."""
    # gphi >= 0: gamma_alpha gamma_theta = 5e-7
    assert ipm.alpha_min_of(0.5, 0.0, 1.0, OPT) == pytest.approx(5e-7, rel=1e-15)
    assert ipm.alpha_min_of(0.5, 3.0, 1.0, OPT) == pytest.approx(5e-7, rel=1e-15)
    # gphi = -2, theta_k = 0.5 > theta_min = 0.1:
    #   min(1e-5, 1e-5 * 0.5 / 2 = 2.5e-6) = 2.5e-6 -> 1.25e-7
    assert ipm.alpha_min_of(0.5, -2.0, 0.1, OPT) == pytest.approx(1.25e-7, rel=1e-14)
    # theta_k = 1e-12 <= theta_min, gphi = -1000: the three candidates are
    #   1e-5;  1e-5 * 1e-12 / 1e3 = 1e-20;  (1e-12)^1.1 / (1e3)^2.3 = 10^-13.2 / 10^6.9 = 10^-20.1
    #   -> 0.05 * 10^-20.1
    assert ipm.alpha_min_of(1e-12, -1000.0, 1.0, OPT) == pytest.approx(0.05 * 10 ** -20.1, rel=1e-12)
    # same theta_k above theta_min: the third candidate does not apply -> 0.05 * 1e-20
    assert ipm.alpha_min_of(1e-12, -1000.0, 1e-13, OPT) == pytest.approx(5e-22, rel=1e-12)


# ---- trial acceptance and the halving sequence ----------------------------------------

def test_first_acceptable_step_of_the_halving_sequence_is_taken():
    """Trials at 1, 1/2, 1/4 increase the infeasibility; the one at 1/8 reduces
    it by half: the search takes alpha = 1/8 after 4 trials (no skipped or
    repeated halving)."""
    seen = []

    def trial(a):
        seen.append(a)
        return (2.0, 5.0) if a > 0.125 else (0.5, 5.0)

    ok, alpha, ftype, trials = ipm.backtrack(trial, 1.0, 1.0, 5.0, -1.0, 1e-4, 1e4, [], OPT)
    assert ok and alpha == 0.125 and trials == 4 and not ftype
    assert seen == [1.0, 0.5, 0.25, 0.125]


def test_trial_inside_the_filter_envelope_is_rejected():
    """Current iterate (theta_k, phi_k) = (1, 20); filter entry (0.5, 10).  The
    trial at alpha = 1, (0.6, 11), decreases theta by 40 % (sufficient decrease
    holds) but lies in the entry's forbidden region theta >= 0.5 and phi >= 10,
    so it is rejected; the trial at 1/2, (0.4, 11), lies left of the entry and is
    taken."""
    filt = [(0.5, 10.0)]
    trial = lambda a: (0.6, 11.0) if a == 1.0 else (0.4, 11.0)
    ok, alpha, ftype, trials = ipm.backtrack(trial, 1.0, 1.0, 20.0, -1.0, 1e-4, 1e4, filt, OPT)
    assert ok and alpha == 0.5 and trials == 2
    # without the entry the first trial is taken
    ok, alpha, _, trials = ipm.backtrack(trial, 1.0, 1.0, 20.0, -1.0, 1e-4, 1e4, [], OPT)
    assert ok and alpha == 1.0 and trials == 1
    # a trial below the entry's phi (9.5 < 10) is outside the envelope too
    assert ipm.trial_acceptable(0.6, 9.5, 1.0, 1.0, 20.0, -1.0, 1e-4, 1e4, filt, OPT) == (True, False)
    # theta_max: a trial with theta >= theta_max is never acceptable
    assert ipm.trial_acceptable(50.0, -1e9, 1.0, 100.0, 20.0, -1.0, 1e-4, 50.0, [], OPT) == (False, False)


def test_switching_condition_selects_the_armijo_test():
    """Almost feasible iterate (theta_k = 1e-6 <= theta_min = 1e-4) with a
    descent direction gphi = -1: at alpha = 1 the switching condition
    1 * 1^2.3 = 1 > (1e-6)^1.1 holds, so the trial must satisfy Armijo,
    phi_t <= phi_k + 1e-4 * alpha * gphi = 5 - 1e-4.  A trial that only reduces
    the infeasibility is rejected there, accepted when theta_k > theta_min."""
    only_feas = (1e-8, 5.0)
    assert ipm.trial_acceptable(*only_feas, 1.0, 1e-6, 5.0, -1.0, 1e-4, 1e4, [], OPT) == (False, True)
    assert ipm.trial_acceptable(*only_feas, 1.0, 1e-6, 5.0, -1.0, 1e-7, 1e4, [], OPT) == (True, False)
    # an Armijo decrease (phi_t = 5 - 2e-4) is an accepted f-type step
    assert ipm.trial_acceptable(1e-6, 5.0 - 2e-4, 1.0, 1e-6, 5.0, -1.0, 1e-4, 1e4, [], OPT) == (True, True)
    # just short of the Armijo bound (5 - 0.5e-4) fails
    assert ipm.trial_acceptable(1e-6, 5.0 - 0.5e-4, 1.0, 1e-6, 5.0, -1.0, 1e-4, 1e4, [], OPT) == (False, True)
    # at a small step the switching condition fails: alpha = 1e-7 gives
    # 1e-7 < (1e-6)^1.1 = 2.5e-7, so sufficient decrease decides (theta 1e-8 < 1e-6)
    assert ipm.trial_acceptable(*only_feas, 1e-7, 1e-6, 5.0, -1.0, 1e-4, 1e4, [], OPT) == (True, False)
    # an ascent direction never switches
    assert ipm.trial_acceptable(*only_feas, 1.0, 1e-6, 5.0, 0.5, 1e-4, 1e4, [], OPT) == (True, False)


def test_line_search_fails_below_alpha_min():
    """No trial is acceptable: the search tries 1, 1/2, ... while alpha >= alpha_min
    and returns the first step below it.  With gphi = -2 and theta_k = 0.5 above
    theta_min, alpha_min = 1.25e-7 (hand-worked above): 2^-22 = 2.38e-7 is the
    last trial (23 trials), 2^-23 = 1.19e-7 ends the search."""
    ok, alpha, ftype, trials = ipm.backtrack(lambda a: (1.0, 100.0), 1.0, 0.5, 1.0, -2.0, 0.1, 1e4,
                                             [], OPT)
    assert not ok
    assert trials == 23 and alpha == 2.0 ** -23
    # a non-finite trial is rejected like any other
    ok, alpha, _, trials = ipm.backtrack(lambda a: (math.nan, math.nan), 0.5, 0.5, 1.0, 1.0, 0.1,
                                         1e4, [], OPT)
    # gphi > 0: alpha_min = 5e-7; 0.5 * 2^-19 = 9.5e-7 is the last trial (20 trials)
    assert not ok and trials == 20 and alpha == 0.5 * 2.0 ** -20


def test_solve_reports_line_search_failure(monkeypatch):
    """When alpha_min exceeds the fraction-to-boundary step (here forced to 2),
    the first line search takes no trial and the solve ends with
    LINESEARCH_FAILED (the paper's "R": no restoration phase) after zero
    accepted iterations."""
    seen = []

    def big_alpha_min(theta_k, gphi, theta_min, opt):
        seen.append((theta_k, gphi))
        return 2.0

    monkeypatch.setattr(ipm, "alpha_min_of", big_alpha_min)
    res = ipm.solve(W.config1())
    assert res.status == ipm.ERR_LINESEARCH
    assert res.iterations == 0 and res.history == []
    assert len(seen) == 1


# ---- bound-multiplier safeguard (Eq. (16)) ------------------------------------------

def test_bound_dual_reset_worked_by_hand():
    """z is clipped into [mu / (kappa s), kappa mu / s]; kappa = 1e10, mu = 0.1."""
    s = np.array([1.0, 1.0, 0.5, 2.0])
    z = np.array([1e12, 1e-15, 0.3, 7.0])
    out = ipm.reset_bound_duals(z, s, 0.1, 1e10)
    # 1e12 > 1e10 * 0.1 / 1 = 1e9 -> 1e9;  1e-15 < 0.1 / 1e10 = 1e-11 -> 1e-11;
    # 0.3 and 7 lie inside their intervals [2e-11, 2e9] and [5e-12, 5e8]
    assert out[0] == pytest.approx(1e9, rel=1e-15)
    assert out[1] == pytest.approx(1e-11, rel=1e-15)
    assert out[2] == 0.3 and out[3] == 7.0


def test_bound_duals_stay_inside_the_safeguard_during_a_solve():
    """After every accepted step s z / mu lies in [1 / kappa, kappa] for each bound."""
    inst = W.small_network(n=3, r=5, N=12, seed=8)
    opt = ipm.Options(kappa_sigma=10.0)
    recs = []
    res = ipm.solve(inst, opt=opt, on_iter=lambda r: recs.append(r["mu"]))
    assert res.iterations > 3
    from oracle.nlp import Problem
    prob = Problem(inst)
    th = res.x[prob.nz:]
    sl, su = th - inst.theta_lo, inst.theta_hi - th
    mu = recs[-1]
    for s, z in ((sl, res.zl), (su, res.zu)):
        ratio = s * z / mu
        assert np.all(ratio >= 1.0 / 10.0 * (1 - 1e-12)) and np.all(ratio <= 10.0 * (1 + 1e-12))
