"""Initial state guess: collocation forward sweep at theta0 (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper initialises the discretised states from a forward solve of the ODE
at the nominal parameters (Section "Optimization framework configurations").
Here the forward solve is the collocation scheme itself, element by element:
``z[0,0] = x0`` (with several experimental conditions, each condition's first
element starts from that condition's x0); ``z[i,0] = sum_j b_j z[i-1,j]``
(``z[i-1,K]`` for Radau nodes); the interior states
``Z = (z[i,1], ..., z[i,K])`` solve the element's K collocation equations
``sum_j D[k][j] z[i,j] - h f(z[i,k], theta) = 0`` by Newton's method started
at ``z[i,k] = z[i,0]``, stopped when ``max|dZ| <= 1e-12 max(1, max|Z|)``
(at most 30 iterations).  An element whose Newton iteration produces a
non-finite value or does not meet the test keeps ``z[i,k] = z[i,0]``.
"""
from __future__ import annotations

import numpy as np


def forward_sweep(prob, theta, tol: float = 1e-12, max_iter: int = 30):
    n, N, K = prob.n, prob.N, prob.K
    D, h = prob.tab.D, prob.h
    z = np.zeros((N, K + 1, n))
    failures = 0
    for i in range(N):
        if i % prob.Nch == 0:   # a condition's first element starts from its x0
            start = prob.x0c[i // prob.Nch].copy()
        z[i, 0] = start
        Z = np.tile(start, (K, 1))                       # [K, n]
        ok = False
        for _ in range(max_iter):
            f = prob.rhs(Z, theta, prob.escale[i])        # [K, n]
            Fz, _ = prob.rhs_jac(Z, theta, prob.escale[i])  # [K, n, n]
            G = np.zeros((K, n))
            Jm = np.zeros((K * n, K * n))
            for k in range(1, K + 1):
                G[k - 1] = D[k, 0] * start - h * f[k - 1]
                for j in range(1, K + 1):
                    G[k - 1] += D[k, j] * Z[j - 1]
                    blk = D[k, j] * np.eye(n)
                    if j == k:
                        blk = blk - h * Fz[k - 1]
                    Jm[(k - 1) * n:k * n, (j - 1) * n:j * n] = blk
            try:
                dZ = np.linalg.solve(Jm, G.reshape(-1)).reshape(K, n)
            except np.linalg.LinAlgError:
                break
            Z = Z - dZ
            if not np.all(np.isfinite(Z)):
                break
            if np.max(np.abs(dZ)) <= tol * max(1.0, np.max(np.abs(Z))):
                ok = True
                break
        if not ok:
            failures += 1
            Z = np.tile(start, (K, 1))
        z[i, 1:] = Z
        start = z[i, K].copy() if prob.radau else prob.tab.b @ z[i]
    return z, failures
