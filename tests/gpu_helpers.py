"""Test-side helpers: oracle iterates and assembly of the documented GPU layouts."""
import numpy as np
import scipy.sparse as sp

from oracle import ipm as oipm
from oracle.nlp import Problem as OProblem


def random_point(oprob, seed, lam_scale=1.0):
    rng = np.random.default_rng(seed)
    inst = oprob.inst
    x = rng.uniform(0.2, 1.2, oprob.n_x)
    lo, hi = inst.theta_lo, inst.theta_hi
    x[oprob.nz:] = lo + (hi - lo) * rng.uniform(0.3, 0.7, oprob.p)
    if inst.logscale:
        x[oprob.nz:] = rng.uniform(-1.0, 0.5, oprob.p)
    lam = lam_scale * rng.standard_normal(oprob.n_c)
    return x, lam


def assemble_J(oprob, out):
    """Sparse constraint Jacobian from the collo_eval layout + implied constants."""
    n, N, p, K = oprob.n, oprob.N, oprob.p, oprob.K
    D, h = oprob.tab.D, oprob.h
    Z = np.arange(oprob.nz).reshape(N, K + 1, n)
    # continuity rows of every element but each experimental condition's first:
    # +1 on z[i][0], -b_j on z[i-1][j] (Radau: -1 on z[i-1][K] only)
    cont = np.array([i for i in range(1, N) if i % oprob.Nch != 0], dtype=np.int64)
    rows, cols, vals = [Z[:, 0].ravel()], [Z[:, 0].ravel()], [np.ones(N * n)]
    for j in range(K + 1):
        b = 1.0 if (oprob.radau and j == K) else (0.0 if oprob.radau else oprob.tab.b[j])
        if b != 0.0:
            rows.append(Z[cont, 0].ravel()); cols.append(Z[cont - 1, j].ravel())
            vals.append(np.full(len(cont) * n, -b))
    for k in range(1, K + 1):
        for j in range(K + 1):
            if j != k:
                rows.append(Z[:, k].ravel()); cols.append(Z[:, j].ravel())
                vals.append(np.full(N * n, D[k, j]))
        R = np.broadcast_to(Z[:, k, :, None], (N, n, n)).ravel()
        Cc = np.broadcast_to(Z[:, k, None, :], (N, n, n)).ravel()
        V = (out["jac_z"][:, k - 1] + D[k, k] * np.eye(n)[None]).ravel()
        rows.append(R); cols.append(Cc); vals.append(V)
        if p:
            R = np.broadcast_to(Z[:, k, :, None], (N, n, p)).ravel()
            Cc = np.broadcast_to(oprob.nz + np.arange(p)[None, None, :], (N, n, p)).ravel()
            rows.append(R); cols.append(Cc); vals.append(out["jac_theta"][:, k - 1].ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(oprob.n_c, oprob.n_x))


def assemble_W(oprob, out):
    n, N, p, K = oprob.n, oprob.N, oprob.p, oprob.K
    Z = np.arange(oprob.nz).reshape(N, K + 1, n)
    rows, cols, vals = [], [], []
    for s in range(n):
        for j in range(K + 1):
            for l in range(K + 1):
                rows.append(Z[:, j, s]); cols.append(Z[:, l, s]); vals.append(out["hess_obj"][:, s, j, l])
    for k in range(1, K + 1):
        R = np.broadcast_to(Z[:, k, :, None], (N, n, n)).ravel()
        Cc = np.broadcast_to(Z[:, k, None, :], (N, n, n)).ravel()
        rows.append(R); cols.append(Cc); vals.append(out["hess_zz"][:, k - 1].ravel())
        if p:
            R = np.broadcast_to(Z[:, k, :, None], (N, n, p)).ravel()
            Cc = np.broadcast_to(oprob.nz + np.arange(p)[None, None, :], (N, n, p)).ravel()
            V = out["hess_ztheta"][:, k - 1].ravel()
            rows += [R, Cc]; cols += [Cc, R]; vals += [V, V]
    rows.append(oprob.nz + np.arange(p)); cols.append(oprob.nz + np.arange(p))
    vals.append(out["hess_thth"])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(oprob.n_x, oprob.n_x))


def rel_max(a, b):
    a = a.toarray() if sp.issparse(a) else np.asarray(a)
    b = b.toarray() if sp.issparse(b) else np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b))))


def sparse_rel(A, B):
    d = (A - B).tocoo()
    m = np.max(np.abs(B.data)) if B.nnz else 1.0
    return float(np.max(np.abs(d.data)) / max(1.0, m)) if d.nnz else 0.0


def newton_system(oprob, x, lam, zl, zu, mu, dw, dc, opt=None):
    """Oracle Newton step and the sigma / rhs the GPU needs for the same system."""
    opt = opt or oipm.Options()
    ev = oprob.evaluate(x, lam)
    dx, dlam, dzl, dzu, inertia, K, fac = oipm.newton_direction(oprob, ev, x, lam, zl, zu, mu, dw,
                                                                dc, opt)
    inst = oprob.inst
    th = x[oprob.nz:]
    sl, su = th - inst.theta_lo, inst.theta_hi - th
    sigma = np.zeros(oprob.n_x)
    sigma[oprob.nz:] = zl / sl + zu / su
    gphi = ev["grad"].copy()
    gphi[oprob.nz:] += -mu / sl + mu / su
    rhs = -np.concatenate([gphi + ev["J"].T @ lam, ev["c"]])
    return dict(ev=ev, sol=np.concatenate([dx, dlam]), inertia=tuple(inertia), sigma=sigma,
                rhs=rhs, K=K)
