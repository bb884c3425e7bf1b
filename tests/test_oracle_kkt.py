"""Pins for the oracle's KKT factorizations: brute-force solves and eigenvalue inertia."""
import dataclasses

import numpy as np
import pytest

from paper_2607_12201_gb300 import workloads as W
from oracle import kkt
from oracle.nlp import Problem


def _kkt(prob, seed, delta_w, delta_c):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.2, 1.0, prob.n_x)
    x[prob.nz:] = rng.uniform(-0.5, 0.5, prob.p) if prob.inst.logscale else rng.uniform(0.2, 1, prob.p)
    lam = rng.standard_normal(prob.n_c)
    ev = prob.evaluate(x, lam)
    sigma = np.zeros(prob.n_x)
    sigma[prob.nz:] = rng.uniform(0.1, 2.0, prob.p)
    return kkt.assemble(ev["J"], ev["W"], sigma, delta_w, delta_c)


CASES = [(lambda: W.small_network(n=2, r=3, N=2, seed=21), 0.0, 1e-8),
         (lambda: W.small_network(n=3, r=4, N=3, seed=22), 1e-3, 1e-6),
         (lambda: W.small_network(n=3, r=5, N=4, seed=23), 0.0, 1e-8),
         (lambda: W.linear_cascade(N=4), 0.0, 1e-8),
         (lambda: W.small_network(n=2, r=3, N=12, seed=24), 1e-4, 1e-8),
         (lambda: W.linear_cascade(N=16), 0.0, 1e-8)]


@pytest.mark.parametrize("scheme", ["radau3", "gauss4"])
@pytest.mark.parametrize("make,dw,dc", CASES)
def test_dense_and_block_match_bruteforce(make, dw, dc, scheme):
    inst = make()
    if scheme == "gauss4":   # continuity couples all K + 1 points of the previous element
        inst = dataclasses.replace(inst, K=4, scheme="gauss")
    prob = Problem(inst)
    K = _kkt(prob, 3, dw, dc)
    A = K.toarray()
    rng = np.random.default_rng(4)
    b = rng.standard_normal(A.shape[0])
    x_ref = np.linalg.solve(A, b)          # partial-pivoting LU, LAPACK gesv
    ev = np.linalg.eigvalsh(A)
    tol_ev = 1e-12 * np.max(np.abs(ev))
    inertia_ref = (int(np.sum(ev > tol_ev)), int(np.sum(ev < -tol_ev)), int(np.sum(np.abs(ev) <= tol_ev)))
    for mode in ["dense", "block"]:
        fac = kkt.factor(K, prob, mode)
        x = kkt.solve(fac, b)
        assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
        assert tuple(fac.inertia) == inertia_ref, (mode, fac.inertia, inertia_ref)


def test_inertia_detects_negative_curvature():
    # KKT of min -x^2 s.t. nothing, bordered: a negative-curvature primal direction
    prob = Problem(W.small_network(n=2, r=3, N=2, seed=31))
    K = _kkt(prob, 5, 0.0, 1e-8)
    A = K.toarray()
    A[prob.nz, prob.nz] -= 1e6            # theta_0 diagonal strongly negative
    import scipy.sparse as sp
    K2 = sp.csr_matrix(A)
    for mode in ["dense", "block"]:
        fac = kkt.factor(K2, prob, mode)
        ev = np.linalg.eigvalsh(A)
        assert fac.inertia == (int(np.sum(ev > 0)), int(np.sum(ev < 0)), 0)
        assert fac.inertia != (prob.n_x, prob.n_c, 0)


def test_inertia_of_D_two_by_two_blocks():
    d = np.array([[1.0, 0, 0, 0], [0, 0.0, 2.0, 0], [0, 2.0, 0.0, 0], [0, 0, 0, -3.0]])
    assert kkt.inertia_of_D(d) == (2, 2, 0)
    d2 = np.array([[2.0, 1.0], [1.0, 2.0]])
    assert kkt.inertia_of_D(d2) == (2, 0, 0)


@pytest.mark.parametrize("make", [
    lambda: W.random_network(4, 8, n_obs=2, M=20, T=5.0, N=33, seed=19),
    lambda: W.random_network(12, 24, n_obs=4, M=20, T=5.0, N=10, seed=43, theta0_spread=0.1),
    lambda: W.linear_cascade(N=50)], ids=["n4_N33", "n12_N10", "cascade_N50"])
def test_bunch_kaufman_inertia_equals_resolved_eigenvalue_count(make):
    """The oracle's inertia (Bunch-Kaufman pivots, Sylvester's law; whole matrix
    or per Schur block, Haynsworth additivity) is the eigenvalue count of the
    whole KKT matrix wherever that count is resolved: every |eigenvalue| above
    1000 n eps ||K||_2, so no rounding error of the eigensolver can move one
    across zero.  The GPU tests compare against the same eigenvalue counts."""
    prob = Problem(make())
    resolved = 0
    for seed, dw in ((3, 0.0), (4, 1e-2), (5, 0.0)):
        K = _kkt(prob, seed, dw, 1e-8)
        ev = np.linalg.eigvalsh(K.toarray())
        if np.min(np.abs(ev)) <= 1000.0 * K.shape[0] * np.finfo(float).eps * np.max(np.abs(ev)):
            continue
        resolved += 1
        want = (int(np.sum(ev > 0)), int(np.sum(ev < 0)), 0)
        for mode in ["dense", "block"]:
            assert tuple(kkt.factor(K, prob, mode).inertia) == want
    assert resolved >= 2
