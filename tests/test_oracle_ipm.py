"""Pins for the oracle's interior-point solve.

The linear-cascade estimation problem discretised by Radau IIA collocation
has an independent reduced-space form: for given theta the discrete states
follow from the Radau IIA Runge-Kutta stage equations (published Butcher
matrix) element by element, and the model output at an observation time is
the cubic through the element's four points.  Minimising the weighted misfit
over theta alone (scipy's Levenberg-Marquardt) must give the same optimum as
the full-space interior-point method.
"""
import math

import numpy as np
import pytest
from scipy.optimize import least_squares

from paper_2607_12201_gb300 import workloads as W
from oracle import ipm
from oracle.nlp import Problem

S6 = math.sqrt(6.0)
C_RADAU = np.array([(4 - S6) / 10, (4 + S6) / 10, 1.0])
A_RADAU = np.array([
    [(88 - 7 * S6) / 360, (296 - 169 * S6) / 1800, (-2 + 3 * S6) / 225],
    [(296 + 169 * S6) / 1800, (88 + 7 * S6) / 360, (-2 - 3 * S6) / 225],
    [(16 - S6) / 36, (16 + S6) / 36, 1.0 / 9.0]])


def reduced_residuals(theta, inst):
    t1, t2 = theta
    A = np.array([[-t1, 0.0], [t1, -t2]])
    h = inst.T / inst.N
    # stage system: Z_k = z0 + h sum_l a_kl A Z_l  ->  (I - h A_rk (x) A) Z = 1 (x) z0
    big = np.eye(6) - h * np.kron(A_RADAU, A)
    z0 = inst.x0.copy()
    pts = []
    for i in range(inst.N):
        Z = np.linalg.solve(big, np.tile(z0, 3)).reshape(3, 2)
        pts.append((z0.copy(), Z))
        z0 = Z[2]
    res = []
    for m in range(inst.M):
        t = inst.obs_t[m]
        i = min(max(int(math.ceil(t * inst.N / inst.T)) - 1, 0), inst.N - 1)
        zs, Z = pts[i]
        ts = i * h + h * np.concatenate([[0.0], C_RADAU])
        vals = np.concatenate([[zs[inst.obs_s[m]]], Z[:, inst.obs_s[m]]])
        yhat = np.polyval(np.polyfit(ts - i * h, vals, 3), t - i * h)
        res.append((yhat - inst.obs_y[m]) / inst.obs_sigma[m])
    return np.array(res)


def test_cascade_ipm_matches_reduced_space_least_squares():
    inst = W.config1()
    ref = least_squares(reduced_residuals, inst.theta0, args=(inst,), xtol=1e-15, ftol=1e-15,
                        gtol=1e-15, method="lm")
    res = ipm.solve(inst, opt=ipm.Options(tol=1e-10))
    assert res.status == ipm.SUCCESS
    prob = Problem(inst)
    th = res.theta(prob)
    assert np.max(np.abs(th - ref.x) / np.abs(ref.x)) < 1e-8, (th, ref.x)
    assert abs(res.phi - 0.5 * np.sum(ref.fun ** 2)) < 1e-8 * res.phi
    # the estimate lands near the data-generating parameters (0.7, 0.3)
    assert np.max(np.abs(th - [0.7, 0.3])) < 0.05


def test_trivial_start_at_optimum_takes_few_iterations():
    # Paper, "Trivial solves": started at the optimum the IPM still iterates,
    # but only to re-centre the barrier.
    inst = W.config1()
    first = ipm.solve(inst)
    th = first.x[-2:]
    again = ipm.solve(inst.with_theta0(th))
    assert again.status == ipm.SUCCESS
    assert again.iterations <= first.iterations
    assert np.max(np.abs(again.x[-2:] - th)) < 1e-5


def test_kkt_conditions_hold_at_solution():
    inst = W.config1()
    res = ipm.solve(inst, opt=ipm.Options(tol=1e-9))
    prob = Problem(inst)
    ev = prob.evaluate(res.x, res.lam)
    dual = ev["grad"] + ev["J"].T @ res.lam
    dual[prob.nz:] += -res.zl + res.zu
    assert np.max(np.abs(dual)) < 1e-8 * max(1.0, np.max(np.abs(res.lam)))
    assert np.max(np.abs(ev["c"])) < 1e-10
    # continuity constraints: z[i,0] = z[i-1,K]
    z, _ = prob.split(res.x)
    assert np.max(np.abs(z[1:, 0] - z[:-1, 3])) < 1e-10


@pytest.mark.slow
def test_small_random_network_converges():
    inst = W.random_network(4, 6, n_obs=4, M=20, T=5.0, N=20, seed=41, theta0_spread=0.1)
    res = ipm.solve(inst)
    assert res.status in (ipm.SUCCESS, ipm.ACCEPTABLE)


# The same reduced-space form for a nonlinear mass-action network: the stage
# equations Z_k = z0 + h sum_l a_kl f(Z_l) of the published Radau IIA Butcher
# matrix, solved by Newton's method element by element, with a hand-written
# mass-action right-hand side f_s = sum_r nu_sr k_r prod_{reactants} z.
def _rate_constants(theta, inst):
    k = np.array(inst.kfix, dtype=float)
    for j in range(inst.r):
        q = inst.pidx[j]
        if q >= 0:
            k[j] = 10.0 ** theta[q] if inst.logscale else theta[q]
    return k


def _mass_action(z, k, inst):
    n = inst.n
    f, J = np.zeros(n), np.zeros((n, n))
    for j in range(inst.r):
        a, b = inst.react[j]
        mon = z[a] * (z[b] if b >= 0 else 1.0)
        dmon = np.zeros(n)
        dmon[a] += z[b] if b >= 0 else 1.0
        if b >= 0:
            dmon[b] += z[a]
        nu = np.zeros(n)
        for s in inst.react[j]:
            if s >= 0:
                nu[s] -= 1.0
        for s in inst.prod[j]:
            if s >= 0:
                nu[s] += 1.0
        f += nu * k[j] * mon
        J += np.outer(nu * k[j], dmon)
    return f, J


def reduced_residuals_network(theta, inst):
    k = _rate_constants(theta, inst)
    n, h = inst.n, inst.T / inst.N
    z0 = np.array(inst.x0, dtype=float)
    pts = []
    for _ in range(inst.N):
        Z = np.tile(z0, (3, 1))
        for _ in range(50):
            fj = [_mass_action(Z[l], k, inst) for l in range(3)]
            F = np.zeros((3, n))
            Jb = np.zeros((3 * n, 3 * n))
            for a in range(3):
                F[a] = Z[a] - z0 - h * sum(A_RADAU[a, l] * fj[l][0] for l in range(3))
                for l in range(3):
                    Jb[a * n:(a + 1) * n, l * n:(l + 1) * n] = \
                        (np.eye(n) if a == l else 0.0) - h * A_RADAU[a, l] * fj[l][1]
            d = np.linalg.solve(Jb, F.reshape(-1)).reshape(3, n)
            Z = Z - d
            if np.max(np.abs(d)) < 1e-15 * max(1.0, np.max(np.abs(Z))):
                break
        pts.append((z0.copy(), Z.copy()))
        z0 = Z[2].copy()
    res = []
    for m in range(inst.M):
        t = inst.obs_t[m]
        i = min(max(int(math.ceil(t * inst.N / inst.T)) - 1, 0), inst.N - 1)
        zs, Z = pts[i]
        s = inst.obs_s[m]
        vals = np.concatenate([[zs[s]], Z[:, s]])
        yhat = np.polyval(np.polyfit(h * np.concatenate([[0.0], C_RADAU]), vals, 3), t - i * h)
        res.append((yhat - inst.obs_y[m]) / inst.obs_sigma[m])
    return np.array(res)


@pytest.mark.parametrize("n,r,seed,theta_rtol", [(3, 4, 7, 1e-7), (4, 6, 41, 1e-6)])
def test_network_ipm_matches_reduced_space_least_squares(n, r, seed, theta_rtol):
    inst = W.random_network(n, r, n_obs=n, M=30, T=5.0, N=12, seed=seed, theta0_spread=0.1)
    ref = least_squares(reduced_residuals_network, inst.theta0, args=(inst,), xtol=1e-15,
                        ftol=1e-15, gtol=1e-15, method="lm")
    res = ipm.solve(inst, opt=ipm.Options(tol=1e-10))
    assert res.status == ipm.SUCCESS
    th = res.theta(Problem(inst))
    assert np.max(np.abs(th - ref.x) / np.abs(ref.x)) < theta_rtol, (th, ref.x)
    assert abs(res.phi - 0.5 * np.sum(ref.fun ** 2)) < 1e-10 * res.phi


def test_noise_free_estimate_converges_at_endpoint_order():
    # With exact data from the closed-form cascade trajectory, the discrete
    # optimum misses theta_true only by the discretisation error at the
    # observation times.  For N = 20, 40, 80 (T = 10) every observation time
    # t_m = m/2 is an element end, where Radau IIA is superconvergent of order
    # 2K - 1 = 5: halving h divides the parameter error by about 2^5.
    errs = []
    for N in (20, 40, 80):
        inst = W.linear_cascade(N=N, noise=False)
        res = ipm.solve(inst, opt=ipm.Options(tol=1e-12))
        assert res.status == ipm.SUCCESS
        errs.append(res.x[-2:] - np.array([0.7, 0.3]))
    for coarse, fine in zip(errs, errs[1:]):
        ratio = np.abs(coarse) / np.abs(fine)
        assert np.all((ratio > 28.0) & (ratio < 36.0)), ratio
        assert np.all(np.sign(coarse) == np.sign(fine))


def test_inertia_correction_follows_the_published_schedule(monkeypatch):
    # Waechter & Biegler (2006), inertia correction: try delta_w = 0; then 1e-4
    # if no earlier iteration needed a correction, else max(delta_min,
    # delta_last / 3); grow by 100 while no correction has ever succeeded, by 8
    # after; remember the accepted value.  The wrapper reports a wrong inertia
    # below a per-iteration threshold and records every delta_w tried.
    thresholds = [0.5, 0.5, None, 1e-3]
    calls = []
    real = ipm.newton_direction

    def fake(prob, ev, x, lam, zl, zu, mu, delta_w, delta_c, opt):
        if delta_w == 0.0:
            calls.append([])
        calls[-1].append(delta_w)
        out = list(real(prob, ev, x, lam, zl, zu, mu, delta_w, delta_c, opt))
        thr = thresholds[len(calls) - 1]
        if thr is not None and delta_w < thr:
            npos, nneg, nzero = out[4]
            out[4] = (npos - 1, nneg + 1, nzero)
        return tuple(out)

    monkeypatch.setattr(ipm, "newton_direction", fake)
    res = ipm.solve(W.config1(), opt=ipm.Options(max_iter=len(thresholds)))
    assert res.iterations == len(thresholds)
    expected = [[0.0, 1e-4, 1e-2, 1.0],                # first correction: x100 from 1e-4
                [0.0, 1.0 / 3.0, 8.0 / 3.0],           # last/3, then x8
                [0.0],                                 # no correction: last value kept
                [0.0, 8.0 / 9.0]]                      # (8/3)/3 suffices
    assert len(calls) == len(expected)
    for got, want in zip(calls, expected):
        assert np.allclose(got, want, rtol=1e-12, atol=0), (got, want)


def test_barrier_parameter_follows_the_monotone_update():
    # Waechter & Biegler (2006), monotone barrier update: whenever the barrier
    # problem is solved to kappa_eps * mu, mu <- max(tol / 10, min(kappa_mu mu,
    # mu^theta_mu)) with kappa_mu = 0.2, theta_mu = 1.5, possibly several times
    # in one iteration.  Every change of mu along the history must be such a
    # chain, mu never grows, and it ends above the floor tol / 10.
    tol = 1e-8
    res = ipm.solve(W.config1(), opt=ipm.Options(tol=tol))
    assert res.status == ipm.SUCCESS
    mus = [h["mu"] for h in res.history]
    assert mus[0] == 0.1
    decreases = 0
    for a, b in zip(mus, mus[1:]):
        assert b <= a
        if b == a:
            continue
        m, steps = a, 0
        while m > b * (1 + 1e-12):
            m = max(tol / 10.0, min(0.2 * m, m ** 1.5))
            steps += 1
        assert abs(m - b) <= 1e-12 * b and steps >= 1, (a, b)
        decreases += steps
    assert decreases >= 4 and min(mus) >= tol / 10.0


def test_fraction_to_boundary_is_the_largest_feasible_step():
    # alpha_max = max{alpha in (0, 1] : v + alpha dv >= (1 - tau) v}, checked
    # against bisection on random cases and two hand-worked ones
    assert ipm.fraction_to_boundary(np.array([1.0]), np.array([-2.0]), 0.99) == 0.495
    assert ipm.fraction_to_boundary(np.array([1.0, 2.0]), np.array([0.5, 3.0]), 0.99) == 1.0
    rng = np.random.default_rng(11)
    for _ in range(200):
        k = int(rng.integers(1, 6))
        v = rng.uniform(1e-3, 2.0, k)
        dv = rng.normal(0.0, 3.0, k)
        tau = rng.uniform(0.9, 0.9999)
        a = ipm.fraction_to_boundary(v, dv, tau)
        feasible = lambda al: np.all(v + al * dv >= (1 - tau) * v - 1e-14)
        assert 0.0 < a <= 1.0 and feasible(a)
        lo, hi = 0.0, 1.0
        if feasible(1.0):
            assert a == 1.0
            continue
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if feasible(mid) else (lo, mid)
        assert abs(a - lo) <= 1e-12 * max(1.0, lo)


def test_initial_parameters_are_pushed_inside_the_bounds():
    # bound push of Waechter & Biegler (2006), Section 3.6: theta0 is moved to at
    # least p_L = min(kappa_1 max(1, |lo|), kappa_2 (hi - lo)) inside the lower
    # bound (p_U likewise), kappa_1 = kappa_2 = 1e-2
    opt = ipm.Options()
    lo, hi = np.full(3, -5.0), np.full(3, 5.0)
    th = ipm.push_into_bounds(np.array([-5.0, 0.3, 7.0]), lo, hi, opt)
    assert np.allclose(th, [-4.95, 0.3, 4.95], rtol=0, atol=1e-15)
    lo, hi = np.full(2, 1e-3), np.full(2, 1e2)
    th = ipm.push_into_bounds(np.array([0.0, 1e3]), lo, hi, opt)
    assert np.allclose(th, [1e-3 + 1e-2, 1e2 - 0.99999], rtol=0, atol=1e-13)


@pytest.mark.parametrize("dw", [0.0, 1e-2])
def test_condensed_step_solves_the_full_primal_dual_newton_system(dw):
    # The oracle solves the augmented system in which the bound duals are folded
    # into Sigma = Z_L / S_L + Z_U / S_U and the barrier gradient; its step, with
    # the bound-dual steps recovered from it, must satisfy every row of the
    # unreduced primal-dual Newton system (Waechter & Biegler 2006, Eq. 11):
    #   (W + dw I) dx + J^T dlam - dzl + dzu = -(grad phi + J^T lam - zl + zu)
    #   J dx - dc dlam = -c
    #   Z_L dth + S_L dzl = mu - S_L zl,   -Z_U dth + S_U dzu = mu - S_U zu
    inst = W.small_network(n=3, r=4, N=5, seed=7)
    prob = Problem(inst)
    rng = np.random.default_rng(5)
    x = rng.uniform(0.2, 1.0, prob.n_x)
    x[prob.nz:] = rng.uniform(-1.0, 0.5, prob.p)
    lam = rng.standard_normal(prob.n_c)
    zl, zu = rng.uniform(0.5, 2.0, prob.p), rng.uniform(0.5, 2.0, prob.p)
    mu, dc = 0.05, 1e-6
    ev = prob.evaluate(x, lam)
    dx, dlam, dzl, dzu, _, _, _ = ipm.newton_direction(prob, ev, x, lam, zl, zu, mu, dw, dc,
                                                       ipm.Options())
    Wm, J = ev["W"].toarray(), ev["J"].toarray()     # W is stored in full (symmetric)
    assert np.array_equal(Wm, Wm.T)
    th = x[prob.nz:]
    sl, su = th - inst.theta_lo, inst.theta_hi - th
    dth = dx[prob.nz:]
    E = np.zeros((prob.n_x, prob.p))
    E[prob.nz:, :] = np.eye(prob.p)
    stat = (Wm + dw * np.eye(prob.n_x)) @ dx + J.T @ dlam - E @ dzl + E @ dzu \
        + (ev["grad"] + J.T @ lam - E @ zl + E @ zu)
    scale = max(1.0, np.max(np.abs(ev["grad"])), np.max(np.abs(J.T @ lam)))
    assert np.max(np.abs(stat)) <= 1e-10 * scale
    assert np.max(np.abs(J @ dx - dc * dlam + ev["c"])) <= 1e-10 * max(1.0, np.max(np.abs(ev["c"])))
    assert np.allclose(zl * dth + sl * dzl, mu - sl * zl, rtol=0, atol=1e-12)
    assert np.allclose(-zu * dth + su * dzu, mu - su * zu, rtol=0, atol=1e-12)


@pytest.mark.parametrize("make", [lambda: W.config1(),
                                  lambda: W.small_network(n=3, r=4, N=6, seed=7)],
                         ids=["cascade", "small_network"])
def test_every_accepted_step_passes_a_filter_acceptance_test(make, monkeypatch):
    # Waechter & Biegler (2006), Section 2.3: a trial point is accepted if it
    # sufficiently reduces the constraint violation theta = ||c||_1 or the
    # barrier function phi_mu against the current iterate (Eq. 18), or, under the
    # switching condition, satisfies the Armijo condition phi_mu(x + alpha d) <=
    # phi_mu(x) + eta_phi alpha grad phi_mu^T d (Eq. 20).  The iterates are taken
    # from the one evaluation per iteration; theta, phi_mu and the step are
    # recomputed from them here.
    inst = make()
    seen = []
    real = Problem.evaluate

    def record(self, x, lam, obj_factor=1.0):
        seen.append(np.array(x, copy=True))
        return real(self, x, lam, obj_factor)

    monkeypatch.setattr(Problem, "evaluate", record)
    res = ipm.solve(inst, opt=ipm.Options(tol=1e-8))
    assert res.status == ipm.SUCCESS
    assert len(seen) == res.iterations + 1
    prob = Problem(inst)
    opt = ipm.Options()
    nz, lo, hi = prob.nz, inst.theta_lo, inst.theta_hi

    def barrier(x, mu):
        th = x[nz:]
        return prob.objective(x)[0] - mu * np.sum(np.log(th - lo)) - mu * np.sum(np.log(hi - th))

    kinds = set()
    for k, rec in enumerate(res.history):
        x0, x1, mu, alpha = seen[k], seen[k + 1], rec["mu"], rec["alpha"]
        th0, th1 = [float(np.sum(np.abs(prob.constraints(v)))) for v in (x0, x1)]
        ph0, ph1 = barrier(x0, mu), barrier(x1, mu)
        d = (x1 - x0) / alpha
        t = x0[nz:]
        g = float(prob.objective(x0)[1] @ d) + float(np.sum((-mu / (t - lo) + mu / (hi - t)) * d[nz:]))
        slack = 1e-12 * max(1.0, abs(ph0))
        by_theta = th1 <= (1 - opt.gamma_theta) * th0 + 1e-14
        by_phi = ph1 <= ph0 - opt.gamma_phi * th0 + slack
        armijo = g < 0 and ph1 <= ph0 + opt.eta_phi * alpha * g + slack
        assert by_theta or by_phi or armijo, k
        kinds.add("theta/phi" if (by_theta or by_phi) else "armijo")
    assert kinds
