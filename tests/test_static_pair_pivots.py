"""The pivot-free elimination the GPU path is built on, checked on the oracle's KKT
systems (CPU).

Paper, Introduction ("pivoting-free factorizable form"): the element unknowns are
ordered as pairs (state z_ij[s], multiplier of constraint row k[s]) -- (z1, c1),
(z2, c2), (z0, c3) in the element interior, (z3, c0) on the interface -- and every
pair is eliminated with its own 2x2 pivot [[w, j], [j, -delta_c]], in a fixed order,
without pivoting; the parameters come last.  The claim: every such pivot (after the
Schur updates of the pairs before it) has one positive and one negative eigenvalue,
so the element blocks contribute inertia (4nN, 4nN) and the inertia of the whole
system is that plus the inertia of the p x p parameter Schur complement.

This test restates that elimination in dense numpy, applies it to the oracle's
regularised KKT matrices at interior-point iterates of three problems and three
regularisations, and checks it against the oracle: the inertia of the same matrix
(Bunch-Kaufman) and the oracle's Newton step.  On the stiff network the inertia check
is against the eigenvalue signs of the whole (small, dense) matrix."""
import numpy as np
import pytest

from paper_2607_12201_gb300 import workloads as W
from oracle import ipm, kkt
from oracle.nlp import Problem


def pair_order(prob):
    n, N, nx = prob.n, prob.N, prob.n_x
    perm = []
    for i in range(N):
        for j, k in ((1, 1), (2, 2), (0, 3), (3, 0)):
            for s in range(n):
                perm += [(i * 4 + j) * n + s, nx + (i * 4 + k) * n + s]
    perm += list(range(prob.nz, nx))
    return np.array(perm)


def static_pair_ldlt(A, b, npairs):
    """2x2-pivot elimination of the first npairs pairs in order, then the rest;
    returns the inertia, the solution and the pivot determinants relative to
    |ad| + b^2 (-1: one positive and one negative eigenvalue, near 0: nearly
    singular, +1 side: definite)."""
    A, b = A.copy(), b.copy()
    pos = neg = 0
    dets = []
    for q in range(npairs):
        lo, hi = 2 * q, 2 * q + 2
        P = A[lo:hi, lo:hi]
        dets.append((P[0, 0] * P[1, 1] - P[0, 1] * P[1, 0]) /
                    (abs(P[0, 0] * P[1, 1]) + P[0, 1] * P[1, 0]))
        ev = np.linalg.eigvalsh(P)
        pos += int(np.sum(ev > 0)); neg += int(np.sum(ev < 0))
        L = A[hi:, lo:hi] @ np.linalg.inv(P)
        A[hi:, hi:] -= L @ A[lo:hi, hi:]
        b[hi:] -= L @ b[lo:hi]
    S = A[2 * npairs:, 2 * npairs:]
    ev = np.linalg.eigvalsh(0.5 * (S + S.T))
    inertia = (pos + int(np.sum(ev > 0)), neg + int(np.sum(ev < 0)), int(np.sum(ev == 0)))
    x = np.zeros(A.shape[0])
    x[2 * npairs:] = np.linalg.solve(S, b[2 * npairs:])
    for q in reversed(range(npairs)):
        lo, hi = 2 * q, 2 * q + 2
        x[lo:hi] = np.linalg.solve(A[lo:hi, lo:hi], b[lo:hi] - A[lo:hi, hi:] @ x[hi:])
    return inertia, x, np.array(dets)


@pytest.mark.parametrize("make", [
    lambda: W.linear_cascade(N=10),
    lambda: W.small_network(n=3, r=4, N=6, seed=7),
    lambda: W.random_network(4, 8, n_obs=3, M=20, T=5.0, N=8, seed=41, theta0_spread=0.1)],
    ids=["cascade", "small_network", "network_n4"])
def test_static_pair_pivots_match_oracle_inertia_and_step(make):
    inst = make()
    prob = Problem(inst)
    perm = pair_order(prob)
    npairs = 4 * prob.n * prob.N
    for iters in (1, 3, 6, 12):
        r = ipm.solve(inst, opt=ipm.Options(max_iter=iters))
        ev = prob.evaluate(r.x, r.lam)
        dc = 1e-8 * r.mu ** 0.25
        th = r.x[prob.nz:]
        sl, su = th - inst.theta_lo, inst.theta_hi - th
        gphi = ev["grad"].copy()
        gphi[prob.nz:] += -r.mu / sl + r.mu / su
        rhs = -np.concatenate([gphi + ev["J"].T @ r.lam, ev["c"]])
        for dw in (0.0, 1e-4, 1.0):
            dx, dlam, _, _, inertia, K, _ = ipm.newton_direction(prob, ev, r.x, r.lam, r.zl, r.zu,
                                                                  r.mu, dw, dc, ipm.Options())
            A = K.toarray()
            ins, xs, dets = static_pair_ldlt(A[np.ix_(perm, perm)], rhs[perm], npairs)
            assert np.all(dets < 0)                      # one +, one - eigenvalue per pair
            assert ins == tuple(kkt.inertia_dense(A))
            sol = np.concatenate([dx, dlam])[perm]
            assert np.max(np.abs(xs - sol)) <= 1e-9 * max(1.0, np.max(np.abs(sol)))


def test_static_pair_pivots_on_the_stiff_network():
    # 30 species, rate constants over six decades: after the Schur updates some
    # pairs become definite (both eigenvalues of one sign; 23 of 480 at the third
    # iterate), so the element blocks are not of inertia (4n, 4n) here -- but no
    # pivot comes near singular and their count equals the eigenvalue count (where,
    # at one of these systems, a Bunch-Kaufman LDL^T of the same matrix is off by
    # one: the smallest eigenvalues are ~1e-9).  Growth without pivoting costs
    # accuracy (1e-4 relative here), which the FP64 refinement of the GPU path
    # recovers.
    inst = W.config3(N=4)
    prob = Problem(inst)
    perm = pair_order(prob)
    npairs = 4 * prob.n * prob.N
    for iters in (1, 3):
        r = ipm.solve(inst, opt=ipm.Options(max_iter=iters))
        ev = prob.evaluate(r.x, r.lam)
        dc = 1e-8 * r.mu ** 0.25
        th = r.x[prob.nz:]
        sl, su = th - inst.theta_lo, inst.theta_hi - th
        gphi = ev["grad"].copy()
        gphi[prob.nz:] += -r.mu / sl + r.mu / su
        rhs = -np.concatenate([gphi + ev["J"].T @ r.lam, ev["c"]])
        for dw in (0.0, 1.0):
            dx, dlam, _, _, inertia, K, _ = ipm.newton_direction(prob, ev, r.x, r.lam, r.zl, r.zu,
                                                                  r.mu, dw, dc, ipm.Options())
            A = K.toarray()
            ins, xs, dets = static_pair_ldlt(A[np.ix_(perm, perm)], rhs[perm], npairs)
            assert np.min(np.abs(dets)) > 1e-6             # no pivot nearly singular
            eig = np.linalg.eigvalsh(A)
            assert ins == (int(np.sum(eig > 0)), int(np.sum(eig < 0)), 0)
            sol = np.concatenate([dx, dlam])[perm]
            assert np.max(np.abs(xs - sol)) <= 1e-3 * max(1.0, np.max(np.abs(sol)))
