"""Filter line-search primal-dual interior-point method (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper solves the collocation NLP with MadNLP, "a filter line-search
interior point solver" (Introduction), at relative KKT tolerance 1e-6 and an
acceptable level 1e-4 reached for 15 iterations (Section "Optimization
framework configurations").  This module states that algorithm in the form
published by Waechter & Biegler (2006), restricted to what the collocation
NLP needs:

* bounds only on theta (states are free), barrier
  ``phi_mu = f - mu sum log(theta - lo) - mu sum log(hi - theta)``;
* monotone barrier update ``mu <- max(tol/10, min(kappa_mu mu, mu^theta_mu))``
  while ``E_mu <= kappa_eps mu``, filter reset on each update;
* Newton step from the augmented KKT system with the inertia correction
  ``delta_w`` (first try 0, then 1e-4 or last/3, grown by 100 or 8) and an
  always-on ``delta_c = 1e-8 mu^(1/4)``;
* fraction-to-boundary ``tau = max(0.99, 1 - mu)`` for primal and bound-dual
  steps; bound duals reset into ``[mu/(k_S s), k_S mu/s]``, ``k_S = 1e10``;
* backtracking (halving) filter line search with the switching condition,
  the Armijo test on ``phi_mu`` and the filter envelope, ``theta = ||c||_1``;
  no second-order correction and no restoration phase (a step below
  ``alpha_min`` ends the solve with LINESEARCH_FAILED, the counterpart of the
  paper's "R" status);
* convergence on the scaled optimality error ``E_0 <= tol`` (s_max = 100),
  or ``E_0 <= acceptable_tol`` for ``acceptable_iter`` consecutive iterations.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import kkt
from .init import forward_sweep
from .nlp import Problem

SUCCESS, ACCEPTABLE = 0, 1
ERR_NUMERIC, ERR_INERTIA, ERR_MAXITER, ERR_LINESEARCH = -3, -4, -5, -7


@dataclasses.dataclass
class Options:
    tol: float = 1e-6
    acceptable_tol: float = 1e-4
    acceptable_iter: int = 15
    max_iter: int = 3000
    mu_init: float = 0.1
    kappa_mu: float = 0.2
    theta_mu: float = 1.5
    kappa_eps: float = 10.0
    tau_min: float = 0.99
    s_max: float = 100.0
    bound_push: float = 1e-2
    bound_frac: float = 1e-2
    kappa_sigma: float = 1e10
    gamma_theta: float = 1e-5
    gamma_phi: float = 1e-5
    delta: float = 1.0
    s_theta: float = 1.1
    s_phi: float = 2.3
    eta_phi: float = 1e-4
    gamma_alpha: float = 0.05
    dw_min: float = 1e-20
    dw_0: float = 1e-4
    dw_max: float = 1e40
    kw_minus: float = 1.0 / 3.0
    kw_plus: float = 8.0
    kw_plus_bar: float = 100.0
    dc_coef: float = 1e-8
    dc_exp: float = 0.25
    kkt_mode: str = "auto"
    refine_sweeps: int = 2


@dataclasses.dataclass
class Result:
    status: int
    iterations: int
    x: np.ndarray
    lam: np.ndarray
    zl: np.ndarray
    zu: np.ndarray
    mu: float
    phi: float
    kkt_error: float
    history: list
    init_failures: int = 0

    def theta(self, prob):
        return self.x[prob.nz:]


def push_into_bounds(theta, lo, hi, opt: Options):
    pl = np.minimum(opt.bound_push * np.maximum(1.0, np.abs(lo)), opt.bound_frac * (hi - lo))
    pu = np.minimum(opt.bound_push * np.maximum(1.0, np.abs(hi)), opt.bound_frac * (hi - lo))
    return np.minimum(np.maximum(theta, lo + pl), hi - pu)


def initial_point(prob: Problem, theta0, opt: Options, x_start=None, lam_start=None):
    """theta0 pushed into the bounds and the forward sweep's states; with a warm
    start x_start the states are its own and theta0 is its theta (pushed)."""
    inst = prob.inst
    if x_start is not None:
        theta0 = np.asarray(x_start, dtype=np.float64)[prob.nz:]
    th = push_into_bounds(np.asarray(theta0, dtype=np.float64), inst.theta_lo, inst.theta_hi, opt)
    if x_start is not None:
        z, fails = np.asarray(x_start, dtype=np.float64)[:prob.nz].copy(), 0
    else:
        z, fails = forward_sweep(prob, th)
    x = np.concatenate([z.reshape(-1), th])
    lam = np.zeros(prob.n_c) if lam_start is None else np.array(lam_start, dtype=np.float64)
    zl = np.ones(prob.p)
    zu = np.ones(prob.p)
    return x, lam, zl, zu, fails


def optimality_error(prob, ev, x, lam, zl, zu, mu, opt: Options):
    """Scaled E_mu of Waechter & Biegler (2006), Eq. (5)."""
    inst = prob.inst
    th = x[prob.nz:]
    sl, su = th - inst.theta_lo, inst.theta_hi - th
    dual = ev["grad"] + ev["J"].T @ lam
    dual[prob.nz:] += -zl + zu
    p, m = prob.p, prob.n_c
    s_d = max(opt.s_max, (np.sum(np.abs(lam)) + np.sum(np.abs(zl)) + np.sum(np.abs(zu)))
              / (m + 2 * p)) / opt.s_max
    s_c = max(opt.s_max, (np.sum(np.abs(zl)) + np.sum(np.abs(zu))) / max(2 * p, 1)) / opt.s_max
    compl = max(np.max(np.abs(sl * zl - mu)) if p else 0.0,
                np.max(np.abs(su * zu - mu)) if p else 0.0)
    return max(np.max(np.abs(dual)) / s_d, np.max(np.abs(ev["c"])), compl / s_c)


def newton_direction(prob, ev, x, lam, zl, zu, mu, delta_w, delta_c, opt: Options):
    """Solve the augmented system at a given iterate and regularisation.

    Returns (dx, dlam, dzl, dzu, inertia, K)."""
    inst = prob.inst
    th = x[prob.nz:]
    sl, su = th - inst.theta_lo, inst.theta_hi - th
    sigma = np.zeros(prob.n_x)
    sigma[prob.nz:] = zl / sl + zu / su
    grad_phi = ev["grad"].copy()
    grad_phi[prob.nz:] += -mu / sl + mu / su
    rhs = -np.concatenate([grad_phi + ev["J"].T @ lam, ev["c"]])
    K = kkt.assemble(ev["J"], ev["W"], sigma, delta_w, delta_c)
    fac = kkt.factor(K, prob, opt.kkt_mode)
    sol = kkt.solve(fac, rhs, opt.refine_sweeps)
    dx, dlam = sol[:prob.n_x], sol[prob.n_x:]
    dth = dx[prob.nz:]
    dzl = mu / sl - zl - (zl / sl) * dth
    dzu = mu / su - zu + (zu / su) * dth
    return dx, dlam, dzl, dzu, fac.inertia, K, fac


def fraction_to_boundary(v, dv, tau):
    """Largest alpha in (0, 1] with v + alpha dv >= (1 - tau) v (v > 0)."""
    alpha = 1.0
    neg = dv < 0
    if np.any(neg):
        alpha = min(alpha, float(np.min(-tau * v[neg] / dv[neg])))
    return alpha


def barrier_value(prob, phi, x, mu):
    inst = prob.inst
    th = x[prob.nz:]
    return phi - mu * np.sum(np.log(th - inst.theta_lo)) - mu * np.sum(np.log(inst.theta_hi - th))


def alpha_min_of(theta_k, gphi, theta_min, opt: Options):
    """Smallest trial step before the line search gives up (Waechter & Biegler
    2006, Eq. (23)), from the current infeasibility theta_k = ||c||_1 and the
    barrier directional derivative gphi."""
    if gphi < 0:
        if theta_k <= theta_min:
            return opt.gamma_alpha * min(opt.gamma_theta, opt.gamma_phi * theta_k / (-gphi),
                                         opt.delta * theta_k ** opt.s_theta / (-gphi) ** opt.s_phi)
        return opt.gamma_alpha * min(opt.gamma_theta, opt.gamma_phi * theta_k / (-gphi))
    return opt.gamma_alpha * opt.gamma_theta


def trial_acceptable(theta_t, phib_t, alpha, theta_k, phi_k, gphi, theta_min, theta_max, filt,
                     opt: Options):
    """Acceptance of one trial point (theta_t = ||c(x_t)||_1, phib_t its barrier
    value) at step alpha: (accepted, ftype).

    Waechter & Biegler (2006): the trial must lie below theta_max and outside
    every filter entry's forbidden region {theta >= theta_f and phi >= phi_f};
    then, if the switching condition (Eq. (19)) holds at an almost feasible
    iterate (theta_k <= theta_min), the Armijo condition on the barrier function
    (Eq. (20); an "f-type" step), else sufficient decrease of either measure
    (Eq. (18))."""
    if not (np.isfinite(theta_t) and np.isfinite(phib_t)):
        return False, False
    if not theta_t < theta_max:
        return False, False
    for (tf, pf) in filt:
        if theta_t >= tf and phib_t >= pf:
            return False, False
    sw = gphi < 0 and alpha * (-gphi) ** opt.s_phi > opt.delta * theta_k ** opt.s_theta
    if theta_k <= theta_min and sw:
        return bool(phib_t <= phi_k + opt.eta_phi * alpha * gphi), True
    return bool(theta_t <= (1.0 - opt.gamma_theta) * theta_k
                or phib_t <= phi_k - opt.gamma_phi * theta_k), False


def backtrack(trial, alpha_max, theta_k, phi_k, gphi, theta_min, theta_max, filt, opt: Options):
    """Backtracking filter line search (Waechter & Biegler 2006, Algorithm A,
    steps A-5.1 to A-5.5, without second-order correction): trial steps
    alpha_max, alpha_max / 2, ... down to alpha_min (Eq. (23)); trial(alpha)
    returns (theta_t, phib_t).  Returns (accepted, alpha, ftype, trials); when
    no trial is accepted alpha is the first step below alpha_min."""
    a_min = alpha_min_of(theta_k, gphi, theta_min, opt)
    alpha = alpha_max
    trials = 0
    while alpha >= a_min:
        trials += 1
        theta_t, phib_t = trial(alpha)
        ok, ftype = trial_acceptable(theta_t, phib_t, alpha, theta_k, phi_k, gphi, theta_min,
                                     theta_max, filt, opt)
        if ok:
            return True, alpha, ftype, trials
        alpha *= 0.5
    return False, alpha, False, trials


def reset_bound_duals(z, s, mu, kappa_sigma):
    """Bound-multiplier safeguard after a step (Waechter & Biegler 2006,
    Eq. (16)): z is kept within [mu / (kappa_sigma s), kappa_sigma mu / s] for
    the slack s of its bound."""
    return np.maximum(np.minimum(z, kappa_sigma * mu / s), mu / (kappa_sigma * s))


def solve(inst, theta0=None, opt: Options | None = None, verbose: bool = False,
          on_iter=None, x_start=None, lam_start=None) -> Result:
    """x_start / lam_start: a warm start (states and theta, multipliers) in
    place of the forward sweep at theta0."""
    opt = opt or Options()
    prob = Problem(inst)
    x, lam, zl, zu, fails = initial_point(prob, inst.theta0 if theta0 is None else theta0, opt,
                                          x_start, lam_start)
    mu = opt.mu_init
    tau = max(opt.tau_min, 1.0 - mu)
    filt = []
    dw_last = 0.0
    acc_count = 0
    c0 = prob.constraints(x)
    th0 = float(np.sum(np.abs(c0)))
    theta_max = 1e4 * max(1.0, th0)
    theta_min = 1e-4 * max(1.0, th0)
    history = []
    status = ERR_MAXITER
    it = 0
    ev = None
    err = math.inf
    while True:
        ev = prob.evaluate(x, lam, 1.0)
        if not (np.isfinite(ev["phi"]) and np.all(np.isfinite(ev["c"]))):
            status = ERR_NUMERIC
            break
        err = optimality_error(prob, ev, x, lam, zl, zu, 0.0, opt)
        if err <= opt.tol:
            status = SUCCESS
            break
        acc_count = acc_count + 1 if err <= opt.acceptable_tol else 0
        if acc_count >= opt.acceptable_iter:
            status = ACCEPTABLE
            break
        if it >= opt.max_iter:
            status = ERR_MAXITER
            break
        # barrier update (monotone Fiacco-McCormick)
        while optimality_error(prob, ev, x, lam, zl, zu, mu, opt) <= opt.kappa_eps * mu:
            new_mu = max(opt.tol / 10.0, min(opt.kappa_mu * mu, mu ** opt.theta_mu))
            if new_mu >= mu:
                break
            mu = new_mu
            tau = max(opt.tau_min, 1.0 - mu)
            filt = []
        # Newton direction with inertia correction
        delta_c = opt.dc_coef * mu ** opt.dc_exp
        want = (prob.n_x, prob.n_c, 0)
        delta_w = 0.0
        dx, dlam, dzl, dzu, inertia, _, _ = newton_direction(prob, ev, x, lam, zl, zu, mu, 0.0,
                                                             delta_c, opt)
        if tuple(inertia) != want:
            delta_w = opt.dw_0 if dw_last == 0.0 else max(opt.dw_min, opt.kw_minus * dw_last)
            while True:
                dx, dlam, dzl, dzu, inertia, _, _ = newton_direction(
                    prob, ev, x, lam, zl, zu, mu, delta_w, delta_c, opt)
                if tuple(inertia) == want:
                    dw_last = delta_w
                    break
                delta_w *= opt.kw_plus_bar if dw_last == 0.0 else opt.kw_plus
                if delta_w > opt.dw_max:
                    break
            if tuple(inertia) != want:
                status = ERR_INERTIA
                break
        # step lengths
        th = x[prob.nz:]
        sl, su = th - inst.theta_lo, inst.theta_hi - th
        dth = dx[prob.nz:]
        alpha_max = min(fraction_to_boundary(sl, dth, tau), fraction_to_boundary(su, -dth, tau))
        alpha_z = min(fraction_to_boundary(zl, dzl, tau), fraction_to_boundary(zu, dzu, tau))
        # filter line search
        theta_k = float(np.sum(np.abs(ev["c"])))
        phi_k = barrier_value(prob, ev["phi"], x, mu)
        gphi = float(ev["grad"] @ dx) + float(np.sum((-mu / sl + mu / su) * dth))

        def trial(alpha):
            xt = x + alpha * dx
            phit, _ = prob.objective(xt)
            thetat = float(np.sum(np.abs(prob.constraints(xt))))
            if not (np.isfinite(phit) and np.isfinite(thetat)):
                return math.nan, math.nan
            return thetat, barrier_value(prob, phit, xt, mu)

        accepted, alpha, ftype, trials = backtrack(trial, alpha_max, theta_k, phi_k, gphi,
                                                   theta_min, theta_max, filt, opt)
        if not accepted:
            status = ERR_LINESEARCH
            break
        if not ftype:
            filt.append(((1.0 - opt.gamma_theta) * theta_k, phi_k - opt.gamma_phi * theta_k))
        x = x + alpha * dx
        lam = lam + alpha * dlam
        zl = zl + alpha_z * dzl
        zu = zu + alpha_z * dzu
        th = x[prob.nz:]
        sl, su = th - inst.theta_lo, inst.theta_hi - th
        zl = reset_bound_duals(zl, sl, mu, opt.kappa_sigma)
        zu = reset_bound_duals(zu, su, mu, opt.kappa_sigma)
        rec = dict(it=it, phi=ev["phi"], inf_pr=float(np.max(np.abs(ev["c"]))), err=err,
                   mu=mu, delta_w=delta_w, alpha=alpha, alpha_z=alpha_z, trials=trials,
                   theta=x[prob.nz:].copy())
        history.append(rec)
        if verbose:
            print(rec)
        if on_iter is not None:
            on_iter(rec)
        it += 1
    phi = float(ev["phi"]) if ev is not None else math.nan
    return Result(status=status, iterations=it, x=x, lam=lam, zl=zl, zu=zu, mu=mu, phi=phi,
                  kkt_error=err, history=history, init_failures=fails)
