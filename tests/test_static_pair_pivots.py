"""The pivot-free elimination the GPU path is built on, checked on the oracle's KKT
systems (CPU).

Paper, Introduction ("pivoting-free factorizable form"): the unknowns of an element
are ordered as pairs (state z_ij[s], multiplier of constraint row k[s]) and every pair
is eliminated with its own 2x2 pivot [[w, j], [j, -delta_c]], in a fixed order, without
pivoting; the parameters come last.  The order is the GPU path's: the interior pairs
of every element, then the chain blocks left over (one pair group per element) in
block-cyclic-reduction order (blocks stride * (2b + 1) for stride = 1, 2, 4, ...,
block 0 last), then the parameters.

* Radau IIA, K = 3 (the GPU path): interior (z1, c1), (z2, c2), (z0, c3); chain
  block (z3, c0) -- the element's end state and its incoming continuity row.
* Gauss-Legendre, K = 4 (the order proposed for that scheme's element): interior
  (z1, c1) .. (z4, c4), the stage system; chain block (z0, c0) -- the element's start
  state and its incoming continuity row z_i0 - sum_j b_j z_(i-1)j, whose Jacobian
  entry is the identity.  The outgoing continuity row touches the whole element, so
  the element's condensation updates its own block's z0 part and the next block's c0
  part; consecutive blocks again couple through one n x n quadrant, so the cyclic
  reduction is the Radau path's.

The claims: every interior pair touches nothing outside its element but its chain
variables and the parameters; on non-stiff problems every pivot (after the Schur
updates of the pairs before it) has one positive and one negative eigenvalue; the
inertia counted from the pivots is that of the matrix and the solution is the
oracle's Newton step.  On the stiff network the inertia check is against the
eigenvalue signs of the whole (small, dense) matrix."""
import dataclasses

import numpy as np
import pytest

from paper_2607_12201_gb300 import workloads as W
from oracle import ipm, kkt
from oracle.nlp import Problem

# (state point, constraint row) groups of the element interior, and of its chain block
SCHEMES = {
    "radau3": dict(interior=((1, 1), (2, 2), (0, 3)), chain=(3, 0)),
    "gauss4": dict(interior=((1, 1), (2, 2), (3, 3), (4, 4)), chain=(0, 0)),
}


def as_scheme(inst, scheme):
    return inst if scheme == "radau3" else dataclasses.replace(inst, K=4, scheme="gauss")


def bcr_block_order(N):
    out, stride = [], 1
    while stride < N:
        out += list(range(stride, N, 2 * stride))
        stride *= 2
    return out + [0]


def group_indices(prob, i, j, k):
    """Flat KKT indices of element i's pairs (z_ij[s], c_ik[s]), s = 0..n-1, interleaved."""
    n, K1 = prob.n, prob.K + 1
    out = []
    for s in range(n):
        out += [(i * K1 + j) * n + s, prob.n_x + (i * K1 + k) * n + s]
    return out


def elimination_order(prob, scheme):
    sch = SCHEMES[scheme]
    perm = []
    for i in range(prob.N):
        for j, k in sch["interior"]:
            perm += group_indices(prob, i, j, k)
    for i in bcr_block_order(prob.N):
        perm += group_indices(prob, i, *sch["chain"])
    perm += list(range(prob.nz, prob.n_x))
    assert sorted(perm) == list(range(prob.n_x + prob.n_c))
    return np.array(perm)


def kkt_systems(inst, iters_list, dws):
    """(prob, regularised KKT matrix, right-hand side, oracle step) at IPM iterates."""
    prob = Problem(inst)
    for iters in iters_list:
        r = ipm.solve(inst, opt=ipm.Options(max_iter=iters))
        ev = prob.evaluate(r.x, r.lam)
        dc = 1e-8 * r.mu ** 0.25
        th = r.x[prob.nz:]
        sl, su = th - inst.theta_lo, inst.theta_hi - th
        gphi = ev["grad"].copy()
        gphi[prob.nz:] += -r.mu / sl + r.mu / su
        rhs = -np.concatenate([gphi + ev["J"].T @ r.lam, ev["c"]])
        for dw in dws:
            dx, dlam, _, _, _, K, _ = ipm.newton_direction(prob, ev, r.x, r.lam, r.zl, r.zu,
                                                            r.mu, dw, dc, ipm.Options())
            yield prob, K.toarray(), rhs, np.concatenate([dx, dlam])


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


NONSTIFF = [
    lambda: W.linear_cascade(N=10),
    lambda: W.small_network(n=3, r=4, N=6, seed=7),
    lambda: W.random_network(4, 8, n_obs=3, M=20, T=5.0, N=8, seed=41, theta0_spread=0.1)]


@pytest.mark.parametrize("scheme", list(SCHEMES))
@pytest.mark.parametrize("make", NONSTIFF, ids=["cascade", "small_network", "network_n4"])
def test_static_pair_pivots_match_oracle_inertia_and_step(make, scheme):
    inst = as_scheme(make(), scheme)
    for prob, A, rhs, sol in kkt_systems(inst, (1, 3, 6, 12), (0.0, 1e-4, 1.0)):
        perm = elimination_order(prob, scheme)
        npairs = (prob.K + 1) * prob.n * prob.N
        ins, xs, dets = static_pair_ldlt(A[np.ix_(perm, perm)], rhs[perm], npairs)
        assert np.all(dets < 0)                      # one +, one - eigenvalue per pair
        assert ins == tuple(kkt.inertia_dense(A))
        sol = sol[perm]
        assert np.max(np.abs(xs - sol)) <= 1e-9 * max(1.0, np.max(np.abs(sol)))


@pytest.mark.parametrize("scheme", list(SCHEMES))
def test_static_pair_pivots_on_the_stiff_network(scheme):
    # 30 species, rate constants over six decades: after the Schur updates some
    # pairs become definite (both eigenvalues of one sign; at the third iterate 21 of
    # 480 Radau pairs, 6 of 600 Gauss pairs), so the element blocks do not split
    # evenly into positive and negative eigenvalues here -- but no pivot comes near
    # singular and their count equals the eigenvalue count.  Growth without pivoting
    # costs accuracy (1e-4 relative for Radau, whose interior system maps the end
    # state back to the start, below 1e-6 for the forward Gauss stage system), which
    # the FP64 refinement of the GPU path recovers.
    inst = as_scheme(W.config3(N=4), scheme)
    for prob, A, rhs, sol in kkt_systems(inst, (1, 3), (0.0, 1.0)):
        perm = elimination_order(prob, scheme)
        npairs = (prob.K + 1) * prob.n * prob.N
        ins, xs, dets = static_pair_ldlt(A[np.ix_(perm, perm)], rhs[perm], npairs)
        assert np.min(np.abs(dets)) > 1e-3             # no pivot nearly singular
        eig = np.linalg.eigvalsh(A)
        assert ins == (int(np.sum(eig > 0)), int(np.sum(eig < 0)), 0)
        sol = sol[perm]
        tol = 1e-3 if scheme == "radau3" else 1e-5
        assert np.max(np.abs(xs - sol)) <= tol * max(1.0, np.max(np.abs(sol)))


@pytest.mark.parametrize("scheme", list(SCHEMES))
def test_element_interior_touches_only_its_chain_variables(scheme):
    """The structure the cyclic reduction relies on.  Every row of an element's
    interior has nonzeros only in that interior, in the chain variables the scheme
    names and in the parameters; and once all interiors are condensed, consecutive
    chain blocks couple through one n x n quadrant only (rows: the later block's
    continuity multipliers; columns: the earlier block's states), non-consecutive
    blocks not at all.  For Gauss the (c_i0, z_i0) quadrant of a chain block stays
    exactly the identity."""
    sch = SCHEMES[scheme]
    inst = as_scheme(W.small_network(n=3, r=4, N=6, seed=7), scheme)
    prob, A, _, _ = next(kkt_systems(inst, (3,), (1e-4,)))
    n, N, K1, nx = prob.n, prob.N, prob.K + 1, prob.n_x
    theta = set(range(prob.nz, nx))
    jc, kc = sch["chain"]

    def zs(i, j):
        return {(i * K1 + j) * n + s for s in range(n)}

    def cs(i, k):
        return {nx + (i * K1 + k) * n + s for s in range(n)} if i < N else set()

    for i in range(N):
        inner = set()
        for j, k in sch["interior"]:
            inner |= zs(i, j) | cs(i, k)
        if scheme == "radau3":   # its own chain block; the next block's continuity row
            allowed = inner | zs(i, jc) | cs(i, kc) | cs(i + 1, kc)
        else:                    # its own start state; the next block's continuity row
            allowed = inner | zs(i, jc) | cs(i + 1, kc)
        for row in inner:
            assert set(np.nonzero(A[row])[0]) <= allowed | theta
    perm = elimination_order(prob, scheme)
    m = len(perm) - 2 * n * N - prob.p
    B = A[np.ix_(perm, perm)]
    S = B[m:, m:] - B[m:, :m] @ np.linalg.solve(B[:m, :m], B[:m, m:])
    pos = {blk: 2 * n * q for q, blk in enumerate(bcr_block_order(N))}

    def z_of(blk):
        return [pos[blk] + 2 * s for s in range(n)]

    def c_of(blk):
        return [pos[blk] + 2 * s + 1 for s in range(n)]

    for a in range(N):
        for b in range(N):
            blk = S[np.ix_(z_of(a) + c_of(a), z_of(b) + c_of(b))]
            if abs(a - b) > 1:
                assert not blk.any()
            elif b == a - 1:                         # rows of block a, columns of block a-1
                assert not blk[:n, :].any() and not blk[:, n:].any()
                assert blk[n:, :n].any()
    if scheme == "gauss4":
        for a in range(N):
            assert np.array_equal(S[np.ix_(c_of(a), z_of(a))], np.eye(n))
