"""Lifted (relaxed-equality) condensed-space interior-point step and solve (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's solver configuration uses MadNLP's "LiftedKKT" form (Section
"Optimization framework configurations"; Introduction: a KKT system brought
into a form that factorizes without pivoting).  Its idea, restated here for
the collocation NLP ``min Phi(x) s.t. c(x) = 0, lo <= theta <= hi``:

* every equality is relaxed to ``-r <= c(x) <= r`` with a small relaxation
  ``r`` and written with a slack: ``c(x) - s = 0``, ``-r <= s <= r``;
* the slacks' bounds carry a barrier and bound duals ``v_l, v_u`` like any
  other bounded variable, so the primal-dual Newton system in
  ``(dx, ds, dlam)`` reads

      [ W + Sigma_x + dw I        0           J^T ] [dx  ]   [r_x]
      [        0           Sigma_s + dw I     -I  ] [ds  ] = [r_s]
      [        J                 -I            0  ] [dlam]   [r_c]

  with ``Sigma_s = v_l / (s + r) + v_u / (r - s) > 0``;
* eliminating ``ds = J dx - r_c`` and ``dlam = (Sigma_s + dw) ds - r_s``
  leaves the condensed primal system

      (W + Sigma_x + dw I + J^T (Sigma_s + dw I) J) dx = r_x + J^T ((Sigma_s + dw) r_c + r_s)

  whose matrix is symmetric positive definite exactly when the full system
  has the inertia (n_x + m, m, 0) an interior-point step needs (eliminate the
  positive slack block, then the negative-definite multiplier block;
  Haynsworth additivity).  So it is factored by Cholesky without pivoting,
  and a failed Cholesky is the inertia-correction signal (grow dw).

Readings (the paper gives no values): the relaxation ``r`` is 1e-8, the
bound-relaxation factor the IPOPT family uses by default (on the linear
cascade the relaxed optimum's theta moves away from the unrelaxed one in
proportion to r: about 5e-7 relative at 1e-8, 8e-5 at 1e-6); no constraint
regularisation ``delta_c`` (the condensed form needs none); refinement on the
unreduced system to 1e-12 relative residual in at most 20 sweeps; everything
else (barrier update, dw schedule, fraction to boundary, filter line search
with theta = ||c(x) - s||_1) is the same Waechter & Biegler (2006) algorithm as
``oracle.ipm``, with the slacks as additional bounded primal variables.

Two factorizations of the condensed matrix, neither in the GPU's order:

* ``DenseCholesky``: the whole matrix dense, ``numpy.linalg.cholesky``;
* ``BlockCholesky``: the natural unknown order (element i's points z_i0..z_iK
  form one group; theta last) is block tridiagonal with a border; eliminated
  group by group (``S_0 = A_00``, ``S_i = A_ii - A_i,i-1 S_{i-1}^{-1} A_i-1,i``,
  border and parameter block as in ``oracle.kkt.BlockFactor``), each ``S_i``
  and the parameter block by ``scipy.linalg.cho_factor``.

Solves are followed by FP64 iterative refinement on the unreduced system.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import ipm as aug
from .ipm import (ACCEPTABLE, ERR_INERTIA, ERR_LINESEARCH, ERR_MAXITER, ERR_NUMERIC, SUCCESS,
                  backtrack, fraction_to_boundary, push_into_bounds, reset_bound_duals)
from .nlp import Problem


@dataclasses.dataclass
class Options(aug.Options):
    relax: float = 1e-8              # r
    lifted_mode: str = "auto"
    lifted_refine_sweeps: int = 20
    lifted_refine_tol: float = 1e-12

    def r(self):
        return self.relax


class NotPositiveDefinite(Exception):
    pass


def condensed_matrix(J, W, sigma_x, sigma_s, delta_w):
    """W + Sigma_x + dw I + J^T (Sigma_s + dw I) J, sparse."""
    Ds = sp.diags(np.asarray(sigma_s, dtype=np.float64) + delta_w)
    H = W + sp.diags(np.asarray(sigma_x, dtype=np.float64) + delta_w)
    return (H + J.T @ Ds @ J).tocsr()


def unreduced_matrix(J, W, sigma_x, sigma_s, delta_w):
    """The full (dx, ds, dlam) system above, sparse."""
    n_c = J.shape[0]
    H = W + sp.diags(np.asarray(sigma_x, dtype=np.float64) + delta_w)
    Ds = sp.diags(np.asarray(sigma_s, dtype=np.float64) + delta_w)
    I = sp.identity(n_c)
    return sp.bmat([[H, None, J.T], [None, Ds, -I], [J, -I, None]], format="csr")


class DenseCholesky:
    def __init__(self, Kc):
        self.Kc = Kc
        try:
            self.L = np.linalg.cholesky(Kc.toarray())
        except np.linalg.LinAlgError as e:
            raise NotPositiveDefinite() from e

    def solve0(self, b):
        y = sla.solve_triangular(self.L, b, lower=True)
        return sla.solve_triangular(self.L, y, lower=True, trans="T")


class BlockCholesky:
    """Natural-order block elimination of the condensed matrix."""

    def __init__(self, Kc, prob):
        self.Kc = Kc
        g = (prob.K + 1) * prob.n
        N, p = prob.N, prob.p
        self.g, self.N, self.p = g, N, p
        Kc = Kc.tocsr()
        blk = lambda a, b: Kc[a * g:(a + 1) * g, b * g:(b + 1) * g].toarray()
        th = slice(N * g, N * g + p)
        self.A_off = [None] + [blk(i, i - 1) for i in range(1, N)]
        self.S_c, self.Bt = [], []
        Sth = Kc[th, th].toarray()
        prev, prev_B = None, None
        try:
            for i in range(N):
                S = blk(i, i)
                B = Kc[i * g:(i + 1) * g, th].toarray()
                if i > 0:
                    A = self.A_off[i]
                    S = S - A @ sla.cho_solve(prev, A.T)
                    B = B - A @ sla.cho_solve(prev, prev_B)
                c = sla.cho_factor(S, lower=True)
                Sth = Sth - B.T @ sla.cho_solve(c, B)
                self.S_c.append(c)
                self.Bt.append(B)
                prev, prev_B = c, B
            self.Sth_c = sla.cho_factor(Sth, lower=True) if p else None
        except np.linalg.LinAlgError as e:
            raise NotPositiveDefinite() from e

    def solve0(self, b):
        g, N, p = self.g, self.N, self.p
        y = [b[i * g:(i + 1) * g].copy() for i in range(N)]
        yth = b[N * g:].copy()
        for i in range(N):
            if i > 0:
                y[i] -= self.A_off[i] @ sla.cho_solve(self.S_c[i - 1], y[i - 1])
            yth -= self.Bt[i].T @ sla.cho_solve(self.S_c[i], y[i])
        xth = sla.cho_solve(self.Sth_c, yth) if p else yth
        x = [None] * N
        for i in reversed(range(N)):
            rhs = y[i] - self.Bt[i] @ xth
            if i + 1 < N:
                rhs -= self.A_off[i + 1].T @ x[i + 1]
            x[i] = sla.cho_solve(self.S_c[i], rhs)
        return np.concatenate(x + [xth])


def factor(Kc, prob, mode="auto"):
    """Cholesky of the condensed matrix; raises NotPositiveDefinite."""
    if mode == "auto":
        mode = "dense" if Kc.shape[0] <= 2500 else "block"
    return DenseCholesky(Kc) if mode == "dense" else BlockCholesky(Kc, prob)


def solve_unreduced(fac, J, sigma_s, delta_w, r_x, r_s, r_c, sweeps: int = 20, M=None,
                    rtol: float = 1e-12):
    """(dx, ds, dlam) of the unreduced system through the condensed factor, with
    FP64 iterative refinement against the unreduced matrix M (if given) until
    ||b - M sol||_inf <= rtol max(1, ||b||_inf) or ``sweeps`` corrections.
    The condensed matrix carries Sigma_s (up to mu / r^2) next to W, so its
    factor is a preconditioner of limited accuracy; refinement on the
    unreduced system restores the step."""
    d = np.asarray(sigma_s, dtype=np.float64) + delta_w

    def once(rx, rs, rc):
        dx = fac.solve0(rx + J.T @ (d * rc + rs))
        ds = J @ dx - rc
        return dx, ds, d * ds - rs

    dx, ds, dl = once(r_x, r_s, r_c)
    if M is not None:
        n_x, m = J.shape[1], J.shape[0]
        b = np.concatenate([r_x, r_s, r_c])
        bn = max(1.0, float(np.max(np.abs(b))))
        for _ in range(sweeps):
            r = b - M @ np.concatenate([dx, ds, dl])
            if not float(np.max(np.abs(r))) > rtol * bn:
                break
            ex, es, el = once(r[:n_x], r[n_x:n_x + m], r[n_x + m:])
            dx, ds, dl = dx + ex, ds + es, dl + el
    return dx, ds, dl


@dataclasses.dataclass
class State:
    x: np.ndarray
    s: np.ndarray
    lam: np.ndarray
    zl: np.ndarray
    zu: np.ndarray
    vl: np.ndarray
    vu: np.ndarray


def slacks_of(prob, st: State, r):
    """Bound distances: theta - lo, hi - theta, s + r, r - s."""
    inst = prob.inst
    th = st.x[prob.nz:]
    return th - inst.theta_lo, inst.theta_hi - th, st.s + r, r - st.s


def initial_point(prob: Problem, theta0, opt: Options, x_start=None, lam_start=None):
    """The augmented method's start (bound push, forward sweep) plus slacks
    s = c(x0) pushed into [-r, r] and unit slack bound duals."""
    x, lam, zl, zu, fails = aug.initial_point(prob, theta0, opt, x_start, lam_start)
    r = opt.r()
    m = prob.n_c
    s = push_into_bounds(prob.constraints(x), np.full(m, -r), np.full(m, r), opt)
    return State(x, s, lam, zl, zu, np.ones(m), np.ones(m)), fails


def optimality_error(prob, ev, st: State, mu, opt: Options):
    """Scaled E_mu of Waechter & Biegler (2006), Eq. (5), with the slacks as
    bounded variables: dual rows for x and s, primal c(x) - s, and
    complementarity of all four bound families."""
    sl, su, vsl, vsu = slacks_of(prob, st, opt.r())
    dual_x = ev["grad"] + ev["J"].T @ st.lam
    dual_x[prob.nz:] += -st.zl + st.zu
    dual_s = -st.lam - st.vl + st.vu
    p, m = prob.p, prob.n_c
    nb = 2 * p + 2 * m
    zsum = np.sum(np.abs(st.zl)) + np.sum(np.abs(st.zu)) + np.sum(np.abs(st.vl)) \
        + np.sum(np.abs(st.vu))
    s_d = max(opt.s_max, (np.sum(np.abs(st.lam)) + zsum) / (m + nb)) / opt.s_max
    s_c = max(opt.s_max, zsum / nb) / opt.s_max
    compl = 0.0
    for d, z in ((sl, st.zl), (su, st.zu), (vsl, st.vl), (vsu, st.vu)):
        if d.size:
            compl = max(compl, float(np.max(np.abs(d * z - mu))))
    dual = max(float(np.max(np.abs(dual_x))), float(np.max(np.abs(dual_s))) if m else 0.0)
    return max(dual / s_d, float(np.max(np.abs(ev["c"] - st.s))), compl / s_c)


def sigmas(prob, st: State, r):
    sl, su, vsl, vsu = slacks_of(prob, st, r)
    sigma_x = np.zeros(prob.n_x)
    sigma_x[prob.nz:] = st.zl / sl + st.zu / su
    return sigma_x, st.vl / vsl + st.vu / vsu


def newton_direction(prob, ev, st: State, mu, delta_w, opt: Options, check_unreduced=False):
    """Condensed-space Newton step at a given iterate and dw.

    Returns a dict with dx, ds, dlam, dzl, dzu, dvl, dvu, or raises
    NotPositiveDefinite when the condensed matrix is not positive definite."""
    r = opt.r()
    sl, su, vsl, vsu = slacks_of(prob, st, r)
    sigma_x, sigma_s = sigmas(prob, st, r)
    grad_phi = ev["grad"].copy()
    grad_phi[prob.nz:] += -mu / sl + mu / su
    r_x = -(grad_phi + ev["J"].T @ st.lam)
    r_s = -(-mu / vsl + mu / vsu - st.lam)
    r_c = -(ev["c"] - st.s)
    Kc = condensed_matrix(ev["J"], ev["W"], sigma_x, sigma_s, delta_w)
    fac = factor(Kc, prob, opt.lifted_mode)
    M = unreduced_matrix(ev["J"], ev["W"], sigma_x, sigma_s, delta_w)
    dx, ds, dlam = solve_unreduced(fac, ev["J"], sigma_s, delta_w, r_x, r_s, r_c,
                                   opt.lifted_refine_sweeps, M, opt.lifted_refine_tol)
    dth = dx[prob.nz:]
    out = dict(dx=dx, ds=ds, dlam=dlam,
               dzl=mu / sl - st.zl - (st.zl / sl) * dth,
               dzu=mu / su - st.zu + (st.zu / su) * dth,
               dvl=mu / vsl - st.vl - (st.vl / vsl) * ds,
               dvu=mu / vsu - st.vu + (st.vu / vsu) * ds,
               sigma_x=sigma_x, sigma_s=sigma_s, r_x=r_x, r_s=r_s, r_c=r_c, Kc=Kc, M=M)
    return out


def barrier_value(prob, phi, x, s, mu, r):
    inst = prob.inst
    th = x[prob.nz:]
    return (phi - mu * np.sum(np.log(th - inst.theta_lo)) - mu * np.sum(np.log(inst.theta_hi - th))
            - mu * np.sum(np.log(s + r)) - mu * np.sum(np.log(r - s)))


def solve(inst, theta0=None, opt: Options | None = None, verbose: bool = False,
          on_iter=None) -> aug.Result:
    """Filter line-search interior-point solve of the relaxed NLP with
    condensed-space steps; same structure and constants as ``oracle.ipm.solve``."""
    opt = opt or Options()
    r = opt.r()
    prob = Problem(inst)
    st, fails = initial_point(prob, inst.theta0 if theta0 is None else theta0, opt)
    mu = opt.mu_init
    tau = max(opt.tau_min, 1.0 - mu)
    filt = []
    dw_last = 0.0
    acc_count = 0
    th0 = float(np.sum(np.abs(prob.constraints(st.x) - st.s)))
    theta_max = 1e4 * max(1.0, th0)
    theta_min = 1e-4 * max(1.0, th0)
    history = []
    status = ERR_MAXITER
    it = 0
    ev = None
    err = math.inf
    while True:
        ev = prob.evaluate(st.x, st.lam, 1.0)
        if not (np.isfinite(ev["phi"]) and np.all(np.isfinite(ev["c"]))):
            status = ERR_NUMERIC
            break
        err = optimality_error(prob, ev, st, 0.0, opt)
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
        while optimality_error(prob, ev, st, mu, opt) <= opt.kappa_eps * mu:
            new_mu = max(opt.tol / 10.0, min(opt.kappa_mu * mu, mu ** opt.theta_mu))
            if new_mu >= mu:
                break
            mu = new_mu
            tau = max(opt.tau_min, 1.0 - mu)
            filt = []
        # Newton direction; a failed Cholesky is the inertia-correction signal
        delta_w = 0.0
        step = None
        try:
            step = newton_direction(prob, ev, st, mu, 0.0, opt)
        except NotPositiveDefinite:
            delta_w = opt.dw_0 if dw_last == 0.0 else max(opt.dw_min, opt.kw_minus * dw_last)
            while True:
                try:
                    step = newton_direction(prob, ev, st, mu, delta_w, opt)
                    dw_last = delta_w
                    break
                except NotPositiveDefinite:
                    delta_w *= opt.kw_plus_bar if dw_last == 0.0 else opt.kw_plus
                    if delta_w > opt.dw_max:
                        break
        if step is None:
            status = ERR_INERTIA
            break
        dx, ds = step["dx"], step["ds"]
        sl, su, vsl, vsu = slacks_of(prob, st, r)
        dth = dx[prob.nz:]
        alpha_max = min(fraction_to_boundary(sl, dth, tau), fraction_to_boundary(su, -dth, tau),
                        fraction_to_boundary(vsl, ds, tau), fraction_to_boundary(vsu, -ds, tau))
        alpha_z = min(fraction_to_boundary(st.zl, step["dzl"], tau),
                      fraction_to_boundary(st.zu, step["dzu"], tau),
                      fraction_to_boundary(st.vl, step["dvl"], tau),
                      fraction_to_boundary(st.vu, step["dvu"], tau))
        theta_k = float(np.sum(np.abs(ev["c"] - st.s)))
        phi_k = barrier_value(prob, ev["phi"], st.x, st.s, mu, r)
        gphi = (float(ev["grad"] @ dx) + float(np.sum((-mu / sl + mu / su) * dth))
                + float(np.sum((-mu / vsl + mu / vsu) * ds)))

        def trial(alpha):
            xt = st.x + alpha * dx
            stt = st.s + alpha * ds
            phit, _ = prob.objective(xt)
            thetat = float(np.sum(np.abs(prob.constraints(xt) - stt)))
            if not (np.isfinite(phit) and np.isfinite(thetat)):
                return math.nan, math.nan
            return thetat, barrier_value(prob, phit, xt, stt, mu, r)

        accepted, alpha, ftype, trials = backtrack(trial, alpha_max, theta_k, phi_k, gphi,
                                                   theta_min, theta_max, filt, opt)
        if not accepted:
            status = ERR_LINESEARCH
            break
        if not ftype:
            filt.append(((1.0 - opt.gamma_theta) * theta_k, phi_k - opt.gamma_phi * theta_k))
        inf_pr = float(np.max(np.abs(ev["c"] - st.s)))
        st = State(st.x + alpha * dx, st.s + alpha * ds, st.lam + alpha * step["dlam"],
                   st.zl + alpha_z * step["dzl"], st.zu + alpha_z * step["dzu"],
                   st.vl + alpha_z * step["dvl"], st.vu + alpha_z * step["dvu"])
        sl, su, vsl, vsu = slacks_of(prob, st, r)
        st.zl = reset_bound_duals(st.zl, sl, mu, opt.kappa_sigma)
        st.zu = reset_bound_duals(st.zu, su, mu, opt.kappa_sigma)
        st.vl = reset_bound_duals(st.vl, vsl, mu, opt.kappa_sigma)
        st.vu = reset_bound_duals(st.vu, vsu, mu, opt.kappa_sigma)
        rec = dict(it=it, phi=ev["phi"], inf_pr=inf_pr, err=err,
                   mu=mu, delta_w=delta_w, alpha=alpha, alpha_z=alpha_z, trials=trials,
                   theta=st.x[prob.nz:].copy())
        history.append(rec)
        if verbose:
            print(rec)
        if on_iter is not None:
            on_iter(rec)
        it += 1
    phi = float(ev["phi"]) if ev is not None else math.nan
    res = aug.Result(status=status, iterations=it, x=st.x, lam=st.lam, zl=st.zl, zu=st.zu, mu=mu,
                     phi=phi, kkt_error=err, history=history, init_failures=fails)
    res.s, res.vl, res.vu = st.s, st.vl, st.vu
    return res
