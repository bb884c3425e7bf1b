"""Simultaneous-method NLP of Eq. 2 / Eq. 3 for mass-action kinetics (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Variables (Eq. 2a): ``x = [z, theta]`` with ``z[i, j, s]`` the state of
species s at interpolation point j of element i (i = 0..N-1, j = 0..K), and
the estimated parameters ``theta[q]``.  Flat index of z[i, j, s] is
``(i*(K+1) + j)*n + s``; theta follows at offset ``nN(K+1)``.

Constraints ``c[i, k, s]`` (same flat layout as z):

* ``k = 0`` (continuity / initial, Eq. 2c / 2d):
  ``c[0,0] = z[0,0] - x0``, ``c[i,0] = z[i,0] - sum_j b_j z[i-1,j]`` for
  i >= 1, with ``b_j = l_j(1)``; for Radau nodes (``b_j = delta_jK``) this is
  ``z[i,0] - z[i-1,K]``, computed as such.
* ``k = 1..K`` (collocation, Eq. 3 with a single experiment):
  ``c[i,k] = sum_j D[k][j] z[i,j] - h f(z[i,k], theta)``.

Mass-action right-hand side: ``f_s = sum_r nu[s,r] k_r prod_{a in R_r} z_a``
with ``nu[s,r] = (#s in products) - (#s in reactants)``; ``k_r = theta_q``
(linear) or ``10**theta_q`` (log10) for an estimated reaction, else fixed.

Objective (Eq. 2a; weighted least squares, the paper only says it penalises
model-measurement deviation): ``Phi = 1/2 sum_m ((yhat_m - y_m)/sigma_m)^2``
with ``yhat_m = sum_j l_j(tau_m) z[i_m, j, s_m]``; element
``i_m = ceil(t_m N / T) - 1`` clamped to [0, N-1], ``tau_m = t_m N / T - i_m``
(a time on an element boundary belongs to the left element, t = 0 to the
first).

Lagrangian (IPOPT sign convention) ``L = obj_factor*Phi + lambda^T c``; its
Hessian is ``W = obj_factor*grad^2 Phi - h sum_{i,k,s} lambda[i,k,s] grad^2 f_s``.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .radau import Tables, basis

LN10 = math.log(10.0)


class Problem:
    """Index bookkeeping and the evaluation routines for one instance."""

    def __init__(self, inst, K: int | None = None):
        K = inst.K if K is None else K
        assert inst.K == K
        self.inst = inst
        self.tab = Tables(K, getattr(inst, "scheme", "radau"))
        self.radau = self.tab.scheme == "radau"
        self.K = K
        self.n, self.r, self.p = inst.n, inst.r, inst.p
        # experimental conditions (Eq. 1d / 2e): condition c's chain of Nch
        # elements is elements c Nch .. (c + 1) Nch - 1; shared theta
        self.Nc = getattr(inst, "Nc", 1)
        self.Nch = inst.N
        self.N = self.Nc * self.Nch
        self.h = inst.T / inst.N
        cx0 = getattr(inst, "cond_x0", None)
        self.x0c = np.asarray(inst.x0 if cx0 is None else cx0, dtype=np.float64).reshape(
            self.Nc, self.n)
        # condition inputs (the lifted p^c of Eq. 3) multiplying each rate
        # constant, per element
        sc = getattr(inst, "cond_scale", None)
        sc = np.ones((self.Nc, self.r)) if sc is None else np.asarray(sc, dtype=np.float64)
        self.escale = np.repeat(sc.reshape(self.Nc, self.r), self.Nch, axis=0)   # [N, r]
        self.starts = np.arange(0, self.N, self.Nch)
        self.nz = self.n * self.N * (K + 1)
        self.n_x = self.nz + self.p
        self.n_c = self.nz
        # stoichiometry nu[s, r]
        self.nu = np.zeros((self.n, self.r))
        for j in range(self.r):
            for s in inst.react[j]:
                if s >= 0:
                    self.nu[s, j] -= 1.0
            for s in inst.prod[j]:
                if s >= 0:
                    self.nu[s, j] += 1.0
        # observation -> (element, tau, basis weights)
        self.obs_elem = np.zeros(inst.M, dtype=np.int64)
        self.obs_w = np.zeros((inst.M, K + 1))
        ocond = getattr(inst, "obs_cond", None)
        for m in range(inst.M):
            u = inst.obs_t[m] * inst.N / inst.T
            i = int(math.ceil(u)) - 1
            i = min(max(i, 0), inst.N - 1)
            self.obs_elem[m] = (0 if ocond is None else int(ocond[m])) * self.Nch + i
            self.obs_w[m] = basis(self.tab.tau, u - i)

    # -- index helpers ------------------------------------------------------
    def zi(self, i, j, s):
        return (i * (self.K + 1) + j) * self.n + s

    def ti(self, q):
        return self.nz + q

    def split(self, x):
        z = x[: self.nz].reshape(self.N, self.K + 1, self.n)
        return z, x[self.nz:]

    # -- rate constants -----------------------------------------------------
    def rate_constants(self, theta):
        """k[r], dk/dtheta[r], d2k/dtheta2[r] (derivative w.r.t. theta_pidx[r])."""
        inst = self.inst
        k = np.array(inst.kfix, dtype=np.float64, copy=True)
        dk = np.zeros(self.r)
        d2k = np.zeros(self.r)
        for j in range(self.r):
            q = inst.pidx[j]
            if q < 0:
                continue
            if inst.logscale:
                k[j] = 10.0 ** theta[q]
                dk[j] = LN10 * k[j]
                d2k[j] = LN10 * LN10 * k[j]
            else:
                k[j] = theta[q]
                dk[j] = 1.0
                d2k[j] = 0.0
        return k, dk, d2k

    # -- monomials prod_{a in R_r} z_a and their derivatives ----------------
    def monomial(self, zn, j):
        """zn: [..., n]. Returns mon [...], list of (species, dmon [...]) and
        list of (species_a, species_b, d2mon scalar) over ordered pairs."""
        slots = [s for s in self.inst.react[j] if s >= 0]
        mon = np.ones(zn.shape[:-1])
        for s in slots:
            mon = mon * zn[..., s]
        grads = []
        for idx, s in enumerate(slots):
            g = np.ones(zn.shape[:-1])
            for idx2, s2 in enumerate(slots):
                if idx2 != idx:
                    g = g * zn[..., s2]
            grads.append((s, g))
        hess = []
        if len(slots) == 2:
            a, b = slots
            hess.append((a, b, 1.0))
            hess.append((b, a, 1.0))
        return mon, grads, hess

    def _scaled(self, k, scale, j):
        """Rate constant k[j] times the condition input of reaction j (scale
        [..., r] broadcast against the node shape, or None: 1)."""
        return k[j] if scale is None else k[j] * scale[..., j]

    def rhs(self, zn, theta, scale=None):
        """f(z, theta) for zn [..., n] -> [..., n]; scale [..., r]: condition inputs."""
        k, _, _ = self.rate_constants(theta)
        f = np.zeros(zn.shape)
        for j in range(self.r):
            mon, _, _ = self.monomial(zn, j)
            f += (self._scaled(k, scale, j) * mon)[..., None] * self.nu[:, j]
        return f

    def rhs_jac(self, zn, theta, scale=None):
        """df/dz [..., n, n] and df/dtheta [..., n, p]."""
        k, dk, _ = self.rate_constants(theta)
        Fz = np.zeros(zn.shape + (self.n,))
        Ft = np.zeros(zn.shape + (self.p,))
        for j in range(self.r):
            mon, grads, _ = self.monomial(zn, j)
            for (t, g) in grads:
                Fz[..., :, t] += (self._scaled(k, scale, j) * g)[..., None] * self.nu[:, j]
            q = self.inst.pidx[j]
            if q >= 0:
                Ft[..., :, q] += (self._scaled(dk, scale, j) * mon)[..., None] * self.nu[:, j]
        return Fz, Ft

    def rhs_hess(self, zn, theta, lam, scale=None):
        """Weighted second derivatives of sum_s lam[..., s] f_s:
        Hzz [..., n, n], Hzt [..., n, p], Htt [p, p] (summed over nodes)."""
        k, dk, d2k = self.rate_constants(theta)
        Hzz = np.zeros(zn.shape + (self.n,))
        Hzt = np.zeros(zn.shape + (self.p,))
        Htt = np.zeros((self.p, self.p))
        for j in range(self.r):
            omega = lam @ self.nu[:, j]          # [...]
            mon, grads, hess = self.monomial(zn, j)
            for (a, b, v) in hess:
                Hzz[..., a, b] += omega * self._scaled(k, scale, j) * v
            q = self.inst.pidx[j]
            if q >= 0:
                for (t, g) in grads:
                    Hzt[..., t, q] += omega * self._scaled(dk, scale, j) * g
                Htt[q, q] += np.sum(omega * self._scaled(d2k, scale, j) * mon)
        return Hzz, Hzt, Htt

    def node_scale(self):
        """Condition inputs broadcast over the K collocation nodes: [N, 1, r]."""
        return self.escale[:, None, :]

    # -- objective ------------------------------------------------------------
    def objective(self, x):
        z, _ = self.split(x)
        inst = self.inst
        phi = 0.0
        g = np.zeros(self.n_x)
        for m in range(inst.M):
            i, s = self.obs_elem[m], inst.obs_s[m]
            yhat = float(self.obs_w[m] @ z[i, :, s])
            res = (yhat - inst.obs_y[m]) / inst.obs_sigma[m]
            phi += 0.5 * res * res
            for j in range(self.K + 1):
                g[self.zi(i, j, s)] += self.obs_w[m, j] * res / inst.obs_sigma[m]
        return phi, g

    def objective_hessian_entries(self):
        rows, cols, vals = [], [], []
        inst = self.inst
        for m in range(inst.M):
            i, s = self.obs_elem[m], inst.obs_s[m]
            w = self.obs_w[m] / inst.obs_sigma[m]
            for j in range(self.K + 1):
                for l in range(self.K + 1):
                    rows.append(self.zi(i, j, s))
                    cols.append(self.zi(i, l, s))
                    vals.append(w[j] * w[l])
        return rows, cols, vals

    # -- constraints ------------------------------------------------------------
    def constraints(self, x):
        z, theta = self.split(x)
        D, h, K = self.tab.D, self.h, self.K
        c = np.zeros((self.N, K + 1, self.n))
        if self.radau:
            c[1:, 0] = z[1:, 0] - z[:-1, K]
        else:
            c[1:, 0] = z[1:, 0] - np.einsum("j,ijs->is", self.tab.b, z[:-1])
        # each condition's first element: its initial condition (Eq. 2d)
        c[self.starts, 0] = z[self.starts, 0] - self.x0c
        f = self.rhs(z[:, 1:, :], theta, self.node_scale())   # [N, K, n]
        for k in range(1, K + 1):
            acc = np.zeros((self.N, self.n))
            for j in range(K + 1):
                acc += D[k, j] * z[:, j, :]
            c[:, k] = acc - h * f[:, k - 1]
        return c.reshape(-1)

    def _zidx(self):
        """Flat z index array [N, K+1, n]."""
        return np.arange(self.nz).reshape(self.N, self.K + 1, self.n)

    def jacobian(self, x):
        z, theta = self.split(x)
        D, h, K, n, N, p = self.tab.D, self.h, self.K, self.n, self.N, self.p
        Fz, Ft = self.rhs_jac(z[:, 1:, :], theta, self.node_scale())   # [N,K,n,n], [N,K,n,p]
        Z = self._zidx()
        rows, cols, vals = [], [], []
        # continuity / initial rows: +I on z[i,0], -b_j I on z[i-1,j] (Radau: -I on
        # z[i-1,K]) except at each condition's first element (initial condition)
        rows.append(Z[:, 0].ravel()); cols.append(Z[:, 0].ravel()); vals.append(np.ones(N * n))
        cont = np.array([i for i in range(1, N) if i % self.Nch != 0], dtype=np.int64)
        if self.radau:
            rows.append(Z[cont, 0].ravel()); cols.append(Z[cont - 1, K].ravel())
            vals.append(-np.ones(len(cont) * n))
        else:
            for j in range(K + 1):
                rows.append(Z[cont, 0].ravel()); cols.append(Z[cont - 1, j].ravel())
                vals.append(np.full(len(cont) * n, -self.tab.b[j]))
        for k in range(1, K + 1):
            for j in range(K + 1):
                if j != k:
                    rows.append(Z[:, k].ravel()); cols.append(Z[:, j].ravel())
                    vals.append(np.full(N * n, D[k, j]))
            # node block D[k][k] I - h dF/dz  (rows s, cols t)
            R = np.broadcast_to(Z[:, k, :, None], (N, n, n))
            C = np.broadcast_to(Z[:, k, None, :], (N, n, n))
            V = -h * Fz[:, k - 1] + D[k, k] * np.eye(n)[None]
            rows.append(R.ravel()); cols.append(C.ravel()); vals.append(V.ravel())
            if p:
                R = np.broadcast_to(Z[:, k, :, None], (N, n, p))
                C = np.broadcast_to(self.nz + np.arange(p)[None, None, :], (N, n, p))
                rows.append(R.ravel()); cols.append(C.ravel()); vals.append((-h * Ft[:, k - 1]).ravel())
        rows, cols, vals = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.n_c, self.n_x))

    def hessian(self, x, lam, obj_factor=1.0):
        """Full symmetric Lagrangian Hessian W as a sparse matrix."""
        z, theta = self.split(x)
        lamr = lam.reshape(self.N, self.K + 1, self.n)
        h, K, n, N, p = self.h, self.K, self.n, self.N, self.p
        Hzz, Hzt, Htt = self.rhs_hess(z[:, 1:, :], theta, lamr[:, 1:, :], self.node_scale())
        Z = self._zidx()
        r0, c0, v0 = self.objective_hessian_entries()
        rows = [np.array(r0, dtype=np.int64)]
        cols = [np.array(c0, dtype=np.int64)]
        vals = [obj_factor * np.array(v0)]
        for k in range(1, K + 1):
            R = np.broadcast_to(Z[:, k, :, None], (N, n, n))
            C = np.broadcast_to(Z[:, k, None, :], (N, n, n))
            rows.append(R.ravel()); cols.append(C.ravel()); vals.append((-h * Hzz[:, k - 1]).ravel())
            if p:
                R = np.broadcast_to(Z[:, k, :, None], (N, n, p))
                C = np.broadcast_to(self.nz + np.arange(p)[None, None, :], (N, n, p))
                V = (-h * Hzt[:, k - 1]).ravel()
                rows += [R.ravel(), C.ravel()]; cols += [C.ravel(), R.ravel()]; vals += [V, V]
        rows.append(self.nz + np.arange(p)); cols.append(self.nz + np.arange(p))
        vals.append(-h * np.diag(Htt))
        rows, cols, vals = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.n_x, self.n_x))

    def evaluate(self, x, lam, obj_factor=1.0):
        phi, g = self.objective(x)
        return dict(phi=phi, grad=obj_factor * g, c=self.constraints(x), J=self.jacobian(x),
                    W=self.hessian(x, lam, obj_factor))
