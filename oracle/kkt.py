"""Regularised primal-dual KKT system: assembly, inertia, solve (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The Newton step of a primal-dual interior-point method for
``min f(x) s.t. c(x) = 0, bounds on x`` solves (Waechter & Biegler 2006,
the augmented system of the filter line-search method the paper's solver
implements; paper Introduction):

    [ W + Sigma + delta_w I     J^T      ] [dx]   [r_x]
    [        J              -delta_c I   ] [dl] = [r_c]

with W the Lagrangian Hessian, J the constraint Jacobian, Sigma the
bound-barrier diagonal.  Unknown order is ``[x (n_x), lambda (n_c)]``.

Two factorizations, chosen to share nothing with the GPU design:

* ``DenseFactor``: the whole matrix dense; inertia from LAPACK's
  Bunch-Kaufman ``sytrf`` (``scipy.linalg.ldl``, Sylvester's law on the block
  diagonal D); solve with partial-pivoting LU.
* ``BlockFactor``: unknowns regrouped element by element
  (``[z_i, lambda_i]`` for i = 0..N-1, then theta) into a block-tridiagonal
  bordered matrix, eliminated in natural order:
  ``S_0 = A_00``, ``S_i = A_ii - A_i,i-1 S_{i-1}^{-1} A_i-1,i``, border
  ``B~_i = B_i - A_i,i-1 S_{i-1}^{-1} B~_{i-1}``, parameter block
  ``S_theta = A_thth - sum_i B~_i^T S_i^{-1} B~_i``.  Each S_i is factored by
  pivoted dense LU; the inertia is the sum of the inertias of the S_i and of
  S_theta (Haynsworth additivity), each from Bunch-Kaufman.

Both solves are followed by FP64 iterative refinement with the sparse matrix.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def assemble(J, W, sigma, delta_w, delta_c):
    n_c, n_x = J.shape
    H = (W + sp.diags(np.asarray(sigma, dtype=np.float64) + delta_w)).tocsr()
    K = sp.bmat([[H, J.T], [J, -delta_c * sp.identity(n_c)]], format="csr")
    return K


def inertia_of_D(d: np.ndarray):
    """(n_pos, n_neg, n_zero) of a block-diagonal (1x1 / 2x2) symmetric D."""
    npos = nneg = nzero = 0
    m = d.shape[0]
    i = 0
    while i < m:
        if i + 1 < m and d[i + 1, i] != 0.0:
            a, b, c = d[i, i], d[i + 1, i], d[i + 1, i + 1]
            det = a * c - b * b
            if det < 0:
                npos += 1; nneg += 1
            elif det > 0:
                if a + c > 0:
                    npos += 2
                else:
                    nneg += 2
            else:
                ev = np.linalg.eigvalsh(np.array([[a, b], [b, c]]))
                npos += int(np.sum(ev > 0)); nneg += int(np.sum(ev < 0)); nzero += int(np.sum(ev == 0))
            i += 2
        else:
            if d[i, i] > 0:
                npos += 1
            elif d[i, i] < 0:
                nneg += 1
            else:
                nzero += 1
            i += 1
    return npos, nneg, nzero


def inertia_dense(A: np.ndarray):
    if A.shape[0] == 0:
        return 0, 0, 0
    _, d, _ = sla.ldl(A, lower=True)
    return inertia_of_D(d)


class DenseFactor:
    def __init__(self, K):
        self.K = K
        A = K.toarray()
        self.inertia = inertia_dense(A)
        self.lu = sla.lu_factor(A)

    def solve0(self, b):
        return sla.lu_solve(self.lu, b)


class BlockFactor:
    """Natural-order block elimination of the element-banded bordered KKT."""

    def __init__(self, K, prob):
        self.K = K
        n, N, Kc, p = prob.n, prob.N, prob.K, prob.p
        nz = prob.nz
        n_x = prob.n_x
        npt = Kc + 1
        perm = []
        for i in range(N):
            zi = np.arange(i * npt * n, (i + 1) * npt * n)
            perm.append(zi)
            perm.append(n_x + zi)
        perm.append(nz + np.arange(p))
        self.perm = np.concatenate(perm)
        self.m = 2 * npt * n
        self.N, self.p = N, p
        Kp = K[self.perm][:, self.perm].tocsr()
        m = self.m
        blk = lambda a, b: Kp[a * m:(a + 1) * m, b * m:(b + 1) * m].toarray()
        th = slice(N * m, N * m + p)
        self.A_off = [None] + [blk(i, i - 1) for i in range(1, N)]   # A_i,i-1
        self.S_lu = []
        self.Bt = []
        inert = np.zeros(3, dtype=np.int64)
        Sth = Kp[th, th].toarray()
        prev_lu = None
        prev_Bt = None
        for i in range(N):
            S = blk(i, i)
            B = Kp[i * m:(i + 1) * m, th].toarray()
            if i > 0:
                A = self.A_off[i]
                S = S - A @ sla.lu_solve(prev_lu, A.T)
                B = B - A @ sla.lu_solve(prev_lu, prev_Bt)
            inert += np.array(inertia_dense(0.5 * (S + S.T)))
            lu = sla.lu_factor(S)
            Sth = Sth - B.T @ sla.lu_solve(lu, B)
            self.S_lu.append(lu)
            self.Bt.append(B)
            prev_lu, prev_Bt = lu, B
        inert += np.array(inertia_dense(0.5 * (Sth + Sth.T)))
        self.Sth_lu = sla.lu_factor(Sth) if p else None
        self.inertia = tuple(int(v) for v in inert)

    def solve0(self, b):
        m, N, p = self.m, self.N, self.p
        bp = b[self.perm]
        y = [bp[i * m:(i + 1) * m].copy() for i in range(N)]
        yth = bp[N * m:].copy()
        for i in range(N):
            if i > 0:
                y[i] -= self.A_off[i] @ sla.lu_solve(self.S_lu[i - 1], y[i - 1])
            yth -= self.Bt[i].T @ sla.lu_solve(self.S_lu[i], y[i])
        xth = sla.lu_solve(self.Sth_lu, yth) if p else yth
        x = [None] * N
        for i in reversed(range(N)):
            rhs = y[i] - self.Bt[i] @ xth
            if i + 1 < N:
                rhs -= self.A_off[i + 1].T @ x[i + 1]
            x[i] = sla.lu_solve(self.S_lu[i], rhs)
        out_p = np.concatenate(x + [xth])
        out = np.empty_like(out_p)
        out[self.perm] = out_p
        return out


def factor(K, prob=None, mode="auto"):
    if mode == "auto":
        mode = "dense" if K.shape[0] <= 2500 else "block"
    return DenseFactor(K) if mode == "dense" else BlockFactor(K, prob)


def solve(fac, b, sweeps: int = 2):
    """Solve K x = b with the factorization and FP64 iterative refinement."""
    x = fac.solve0(b)
    for _ in range(sweeps):
        r = b - fac.K @ x
        x = x + fac.solve0(r)
    return x
