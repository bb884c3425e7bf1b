"""Why the element and reduction factorizations do not use TF32 tensor cores:
a CPU emulation on the oracle's KKT systems.

The GPU's static-pair elimination (the order of tests/test_static_pair_pivots.py:
element interiors, chain blocks in cyclic-reduction order, parameters last) is
replayed in FP32 with every Schur update either in FP32 or with its operands
rounded to TF32 (10-bit mantissa, round to nearest even) and accumulated in FP32,
the product a tensor core would form; the p x p parameter block is kept and
factored in FP64 as on the GPU.  FP64 iterative refinement with the exact
matrix then needs 1-2 sweeps from the FP32 factor to reach a relative residual
of 1e-10, but 6 to 39 from the TF32 one, or diverges.  Every refinement sweep
is a solve (an HBM-bound pass over the factor), and a step whose refinement
fails is redone in FP64, so TF32 would cost more than it saves.  Splitting
each operand into two TF32 parts and forming three TF32 products per update
(hi·hi + hi·lo + lo·hi, FP32 accumulation) brings the sweeps back to the FP32
count: FP32-accurate updates from tensor cores cost three MMAs per product.
"""
import numpy as np
import pytest

from paper_2607_12201_gb300 import workloads as W
from oracle import ipm
from oracle.nlp import Problem
from gpu_helpers import newton_system
from test_static_pair_pivots import elimination_order


def to_tf32(a):
    """Round float32 values to TF32 (10 explicit mantissa bits), nearest even."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0xFFF + ((u >> 13) & 1)) >> 13) << 13
    return u.astype(np.uint32).view(np.float32)


def split3_product(Lb, Xt):
    """Lb @ Xt from three TF32 products (the split form a tensor core can run
    at FP32 accuracy): hi_L hi_X + hi_L lo_X + lo_L hi_X, with hi = tf32(v) and
    lo = tf32(v - hi), accumulated in FP32."""
    Lh = to_tf32(Lb)
    Ll = to_tf32(Lb - Lh)
    Xh = to_tf32(Xt)
    Xl = to_tf32(Xt - Xh)
    return Lh @ Xh + Lh @ Xl + Ll @ Xh


def static_factor(Kp, npairs, tf32):
    """L (unit lower) and block-diagonal D of the pair-by-pair elimination of the
    permuted matrix in FP32; the trailing parameter block is left in D (FP64).
    tf32: False (FP32 products), True (TF32 products) or "split3"."""
    A = Kp.astype(np.float32)
    m = A.shape[0]
    L = np.eye(m)
    D = np.zeros((m, m))
    c = 0
    for _ in range(npairs):
        P = A[c:c + 2, c:c + 2].astype(np.float64)
        D[c:c + 2, c:c + 2] = P
        X = A[c + 2:, c:c + 2]
        Lb = (X.astype(np.float64) @ np.linalg.inv(P)).astype(np.float32)
        L[c + 2:, c:c + 2] = Lb
        if tf32 == "split3":
            upd = split3_product(Lb, np.ascontiguousarray(X.T))
        else:
            upd = (to_tf32(Lb) @ to_tf32(X.T)) if tf32 else (Lb @ X.T)
        A[c + 2:, c + 2:] -= upd
        c += 2
    D[c:, c:] = A[c:, c:].astype(np.float64)
    return L, D


def refinement_sweeps(K, b, L, D, perm, tol=1e-10, maxit=60):
    def solve(rhs):
        y = np.linalg.solve(L.T, np.linalg.solve(D, np.linalg.solve(L, rhs[perm])))
        out = np.empty_like(y)
        out[perm] = y
        return out
    x = solve(b)
    for k in range(maxit + 1):
        r = b - K @ x
        if not np.all(np.isfinite(r)):
            return None
        if np.max(np.abs(r)) / max(1.0, np.max(np.abs(b))) <= tol:
            return k
        x = x + solve(r)
    return None


@pytest.mark.parametrize("make", [
    lambda: W.random_network(9, 18, n_obs=4, M=20, T=5.0, N=20, seed=6002, theta0_spread=0.1),
    lambda: W.random_network(14, 28, n_obs=4, M=20, T=5.0, N=8, seed=6003, theta0_spread=0.1)],
    ids=["n9_N20", "n14_N8"])
def test_tf32_schur_updates_break_fp64_refinement(make):
    inst = make()
    prob = Problem(inst)
    x, lam, zl, zu, _ = ipm.initial_point(prob, inst.theta0, ipm.Options())
    ref = newton_system(prob, x, lam, zl, zu, 0.1, 1e-3, 1e-8 * 0.1 ** 0.25)
    K, b = ref["K"].toarray(), ref["rhs"]
    perm = elimination_order(prob, "radau3")
    Kp = K[np.ix_(perm, perm)]
    npairs = prob.nz   # (state, multiplier) pairs: n_c of them
    k32 = refinement_sweeps(K, b, *static_factor(Kp, npairs, False), perm)
    ktf = refinement_sweeps(K, b, *static_factor(Kp, npairs, True), perm)
    assert k32 is not None and k32 <= 3
    assert ktf is None or ktf >= 3 * max(k32, 1)
    # three TF32 products per update (split operands) recover the FP32 sweeps
    k3 = refinement_sweeps(K, b, *static_factor(Kp, npairs, "split3"), perm)
    assert k3 is not None and k3 <= k32 + 1
