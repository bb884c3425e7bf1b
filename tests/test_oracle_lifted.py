"""Pins for the oracle's lifted (relaxed-equality) condensed-space method.

* The condensed step against a brute-force dense solve of the whole
  linearised primal-dual system of the relaxed problem (x, slacks,
  multipliers and all four families of bound duals), written row by row from
  the optimality conditions (Waechter & Biegler 2006, Eq. (4) with the
  slacks as bounded variables).
* The same step through a different elimination: eliminating only the slack
  block leaves the augmented system with a per-row constraint diagonal
  -(Sigma_s + dw)^-1, solved by ``oracle.kkt``'s pivoted LU.
* Positive definiteness of the condensed matrix against the eigenvalues of
  the unreduced matrix: Cholesky succeeds exactly when those have the inertia
  (n_x + m, m, 0).
* The block (natural-order) and dense Cholesky factorizations agree.
* As the relaxation r goes to 0 the relaxed optimum tends to the unrelaxed
  one: on the linear cascade, against the independent reduced-space
  least-squares optimum (Radau IIA stage equations), with the gap shrinking
  in proportion to r.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import least_squares

from paper_2607_12201_gb300 import workloads as W
from oracle import ipm, kkt, lifted
from oracle.nlp import Problem
from test_oracle_ipm import reduced_residuals


def _state(prob, opt, seed, lam_scale=0.5):
    rng = np.random.default_rng(seed)
    inst = prob.inst
    x = rng.uniform(0.2, 1.2, prob.n_x)
    lo, hi = inst.theta_lo, inst.theta_hi
    x[prob.nz:] = lo + (hi - lo) * rng.uniform(0.3, 0.7, prob.p)
    if inst.logscale:
        x[prob.nz:] = rng.uniform(-1.0, 0.5, prob.p)
    m = prob.n_c
    r = opt.r()
    return lifted.State(x=x, s=r * rng.uniform(-0.9, 0.9, m),
                        lam=lam_scale * rng.standard_normal(m),
                        zl=rng.uniform(0.5, 2.0, prob.p), zu=rng.uniform(0.5, 2.0, prob.p),
                        vl=rng.uniform(0.5, 2.0, m), vu=rng.uniform(0.5, 2.0, m))


def _tiny():
    return W.small_network(n=2, r=3, N=3, seed=17)


@pytest.mark.parametrize("relax", [1e-2, 1e-8])
@pytest.mark.parametrize("dw", [0.0, 3.0])
def test_condensed_step_solves_the_whole_primal_dual_system(relax, dw):
    inst = _tiny()
    prob = Problem(inst)
    opt = lifted.Options(relax=relax)
    st = _state(prob, opt, 5)
    mu = 0.03
    ev = prob.evaluate(st.x, st.lam)
    try:
        step = lifted.newton_direction(prob, ev, st, mu, dw, opt)
    except lifted.NotPositiveDefinite:
        pytest.skip("condensed matrix not positive definite at this point")
    n_x, m, p, nz = prob.n_x, prob.n_c, prob.p, prob.nz
    r = relax
    J, Wh = ev["J"].toarray(), ev["W"].toarray()
    th = st.x[nz:]
    sl, su = th - inst.theta_lo, inst.theta_hi - th
    E = np.zeros((n_x, p))
    E[nz:, :] = np.eye(p)
    # unknown blocks: dx, ds, dlam, dzl, dzu, dvl, dvu
    sizes = [n_x, m, m, p, p, m, m]
    off = np.concatenate([[0], np.cumsum(sizes)])
    T = off[-1]
    A = np.zeros((T, T))
    b = np.zeros(T)
    X, S, LA, ZL, ZU, VL, VU = [slice(off[k], off[k + 1]) for k in range(7)]
    R = [slice(off[k], off[k + 1]) for k in range(7)]
    # stationarity in x: grad Phi + J^T lam - E zl + E zu = 0
    A[R[0], X] = Wh + dw * np.eye(n_x)
    A[R[0], LA] = J.T
    A[R[0], ZL] = -E
    A[R[0], ZU] = E
    b[R[0]] = -(ev["grad"] + J.T @ st.lam - E @ st.zl + E @ st.zu)
    # stationarity in s: -lam - vl + vu = 0
    A[R[1], S] = dw * np.eye(m)
    A[R[1], LA] = -np.eye(m)
    A[R[1], VL] = -np.eye(m)
    A[R[1], VU] = np.eye(m)
    b[R[1]] = -(-st.lam - st.vl + st.vu)
    # primal: c(x) - s = 0
    A[R[2], X] = J
    A[R[2], S] = -np.eye(m)
    b[R[2]] = -(ev["c"] - st.s)
    # complementarity: (theta - lo) zl = mu, (hi - theta) zu = mu,
    # (s + r) vl = mu, (r - s) vu = mu
    A[R[3], X] = np.diag(st.zl) @ E.T
    A[R[3], ZL] = np.diag(sl)
    b[R[3]] = mu - sl * st.zl
    A[R[4], X] = -np.diag(st.zu) @ E.T
    A[R[4], ZU] = np.diag(su)
    b[R[4]] = mu - su * st.zu
    A[R[5], S] = np.diag(st.vl)
    A[R[5], VL] = np.diag(st.s + r)
    b[R[5]] = mu - (st.s + r) * st.vl
    A[R[6], S] = -np.diag(st.vu)
    A[R[6], VU] = np.diag(r - st.s)
    b[R[6]] = mu - (r - st.s) * st.vu
    u = np.linalg.solve(A, b)
    got = np.concatenate([step[k] for k in ("dx", "ds", "dlam", "dzl", "dzu", "dvl", "dvu")])
    for k, name in enumerate(("dx", "ds", "dlam", "dzl", "dzu", "dvl", "dvu")):
        ref = u[off[k]:off[k + 1]]
        scale = max(np.max(np.abs(u)), 1.0)
        assert np.max(np.abs(step[name] - ref)) <= 2e-8 * scale, name
    assert got.shape == u.shape


def test_condensed_step_equals_the_augmented_solve_with_a_row_diagonal():
    """Eliminating only the slack block: [[H, J^T], [J, -(Sigma_s+dw)^-1]]
    [dx; dlam] = [r_x; r_c + (Sigma_s+dw)^-1 r_s], solved by pivoted LU."""
    inst = W.small_network(n=3, r=4, N=4, seed=7)
    prob = Problem(inst)
    opt = lifted.Options(relax=1e-4)
    st = _state(prob, opt, 9, lam_scale=0.1)
    mu, dw = 0.01, 1.0
    ev = prob.evaluate(st.x, st.lam)
    step = lifted.newton_direction(prob, ev, st, mu, dw, opt)
    d = step["sigma_s"] + dw
    H = ev["W"] + sp.diags(step["sigma_x"] + dw)
    Kaug = sp.bmat([[H, ev["J"].T], [ev["J"], -sp.diags(1.0 / d)]], format="csr")
    rhs = np.concatenate([step["r_x"], step["r_c"] + step["r_s"] / d])
    fac = kkt.DenseFactor(Kaug)
    sol = kkt.solve(fac, rhs, sweeps=2)
    n_x = prob.n_x
    assert np.max(np.abs(sol[:n_x] - step["dx"])) <= 1e-9 * max(1.0, np.max(np.abs(sol[:n_x])))
    assert np.max(np.abs(sol[n_x:] - step["dlam"])) <= 1e-9 * max(1.0, np.max(np.abs(sol[n_x:])))
    assert fac.inertia == (n_x, prob.n_c, 0)


@pytest.mark.parametrize("seed", [1, 2, 5, 8])
def test_cholesky_succeeds_exactly_when_the_unreduced_inertia_is_right(seed):
    """Large multipliers make W indefinite; sweep dw across the transition."""
    inst = _tiny()
    prob = Problem(inst)
    opt = lifted.Options(relax=1e-3)
    st = _state(prob, opt, seed, lam_scale=30.0)
    ev = prob.evaluate(st.x, st.lam)
    sx, ss = lifted.sigmas(prob, st, opt.r())
    n_x, m = prob.n_x, prob.n_c
    seen = set()
    for dw in [0.0, 1e-3, 1e-1, 1.0, 10.0, 100.0, 1e3, 1e4]:
        M = lifted.unreduced_matrix(ev["J"], ev["W"], sx, ss, dw).toarray()
        ev_ = np.linalg.eigvalsh(M)
        right = int(np.sum(ev_ > 0)) == n_x + m and int(np.sum(ev_ < 0)) == m
        Kc = lifted.condensed_matrix(ev["J"], ev["W"], sx, ss, dw)
        try:
            lifted.DenseCholesky(Kc)
            ok = True
        except lifted.NotPositiveDefinite:
            ok = False
        assert ok == right, dw
        try:
            lifted.BlockCholesky(Kc, prob)
            okb = True
        except lifted.NotPositiveDefinite:
            okb = False
        assert okb == right, dw
        seen.add(ok)
    assert seen == {True, False}


def test_block_and_dense_cholesky_solve_alike():
    inst = W.small_network(n=3, r=5, N=7, seed=8)
    prob = Problem(inst)
    opt = lifted.Options(relax=1e-6)
    st = _state(prob, opt, 3, lam_scale=0.1)
    ev = prob.evaluate(st.x, st.lam)
    sx, ss = lifted.sigmas(prob, st, opt.r())
    Kc = lifted.condensed_matrix(ev["J"], ev["W"], sx, ss, 1.0)
    b = np.random.default_rng(0).standard_normal(prob.n_x)
    xd = lifted.DenseCholesky(Kc).solve0(b)
    xb = lifted.BlockCholesky(Kc, prob).solve0(b)
    assert np.max(np.abs(xd - xb)) <= 1e-8 * max(1.0, np.max(np.abs(xd)))
    assert np.max(np.abs(Kc @ xb - b)) <= 1e-6 * np.max(np.abs(b)) * np.max(np.abs(Kc.data))


def test_relaxed_optimum_tends_to_the_reduced_space_optimum():
    inst = W.config1()
    ref = least_squares(reduced_residuals, inst.theta0, args=(inst,), xtol=1e-15, ftol=1e-15,
                        gtol=1e-15, method="lm")
    gaps = {}
    for r in (1e-7, 1e-8, 1e-10):
        res = lifted.solve(inst, opt=lifted.Options(relax=r, tol=1e-9))
        assert res.status == ipm.SUCCESS, r
        th = res.x[-inst.p:]
        gaps[r] = float(np.max(np.abs(th - ref.x) / np.abs(ref.x)))
        # relaxed constraints: every slack inside [-r, r], c(x) = s to the tolerance
        prob = Problem(inst)
        assert np.max(np.abs(res.s)) <= r
        assert np.max(np.abs(prob.constraints(res.x) - res.s)) <= 1e-9
    assert gaps[1e-10] <= 1e-7
    # first order in r: ten times the relaxation, about ten times the gap
    assert 3.0 <= gaps[1e-7] / gaps[1e-8] <= 30.0


def test_lifted_measures_are_those_of_the_slack_nlp_in_standard_form():
    """The relaxed problem is a standard-form NLP in X = (z, theta, s) with
    bounds on (theta, s) and constraints c(x) - s = 0.  Its scaled optimality
    error and barrier function, computed by the pinned augmented-form
    routines (``oracle.ipm``) on that NLP, equal the lifted routines' values."""
    import types
    inst = W.small_network(n=3, r=4, N=5, seed=7)
    prob = Problem(inst)
    opt = lifted.Options(relax=1e-3)
    st = _state(prob, opt, 17, lam_scale=2.0)
    ev = prob.evaluate(st.x, st.lam)
    r, m, p = opt.r(), prob.n_c, prob.p
    fake_inst = types.SimpleNamespace(theta_lo=np.concatenate([inst.theta_lo, np.full(m, -r)]),
                                      theta_hi=np.concatenate([inst.theta_hi, np.full(m, r)]))
    fake = types.SimpleNamespace(inst=fake_inst, nz=prob.nz, p=p + m, n_c=m,
                                 n_x=prob.n_x + m)
    X = np.concatenate([st.x, st.s])
    ev_std = {"grad": np.concatenate([ev["grad"], np.zeros(m)]),
              "J": sp.hstack([ev["J"], -sp.identity(m)]).tocsr(),
              "c": ev["c"] - st.s}
    zl = np.concatenate([st.zl, st.vl])
    zu = np.concatenate([st.zu, st.vu])
    for mu in (0.0, 0.07):
        e_std = ipm.optimality_error(fake, ev_std, X, st.lam, zl, zu, mu, opt)
        e_lift = lifted.optimality_error(prob, ev, st, mu, opt)
        assert abs(e_std - e_lift) <= 1e-12 * max(1.0, e_std)
        b_std = ipm.barrier_value(fake, ev["phi"], X, 0.07)
        b_lift = lifted.barrier_value(prob, ev["phi"], st.x, st.s, 0.07, r)
        assert abs(b_std - b_lift) <= 1e-12 * max(1.0, abs(b_std))


def test_lifted_start_pushes_the_slacks_like_any_bounded_variable():
    inst = W.small_network(n=3, r=4, N=5, seed=7)
    prob = Problem(inst)
    opt = lifted.Options(relax=1e-3)
    st, _ = lifted.initial_point(prob, inst.theta0, opt)
    r = opt.r()
    c = prob.constraints(st.x)
    assert np.array_equal(st.s, ipm.push_into_bounds(c, np.full(c.size, -r), np.full(c.size, r),
                                                     opt))
    assert np.all(st.vl == 1.0) and np.all(st.vu == 1.0) and not np.any(st.lam)
