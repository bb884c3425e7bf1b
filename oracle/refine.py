"""Mesh refinement: collocation defect, interpolation onto a finer mesh and
the refine-and-resolve loop (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper names refinement of the interval width, in an outer loop, as the
remedy for a collocation mesh that is too coarse near the optimum (Section
"Static collocation mesh limitations"; Conclusion).  Stated plainly:

* defect of element i: the collocation polynomial
  ``z_i(tau) = sum_j l_j(tau) z_ij`` evaluated at the midpoints
  ``tau*_m = (tau_(m-1) + tau_m) / 2`` (m = 1..K) of consecutive interpolation
  points leaves ``d_ims = sum_j l_j'(tau*_m) z_ijs - h f_s(z_i(tau*_m), theta)``;
  the element's defect is ``max_{m,s} |d_ims|``;
* interpolation: the states of a finer mesh at ``t = (i + tau_j) h_f`` from
  the coarse polynomial of the element holding t (a time on an element
  boundary from the left element, t = 0 from the first), theta copied;
* loop: solve; while the solve converged, the defect exceeds the tolerance
  and the doubled mesh is allowed, solve again on twice as many elements
  from the interpolated solution (multipliers zero).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import ipm
from .nlp import Problem
from .radau import basis


def basis_derivative(tau, t):
    """l_j'(t) for j = 0..K: the derivative of prod_{m != j} (t - tau_m) / (tau_j - tau_m)."""
    K1 = len(tau)
    out = np.zeros(K1)
    for j in range(K1):
        for a in range(K1):
            if a == j:
                continue
            term = 1.0 / (tau[j] - tau[a])
            for m in range(K1):
                if m != j and m != a:
                    term *= (t - tau[m]) / (tau[j] - tau[m])
            out[j] += term
    return out


def residual_at(prob: Problem, x, points):
    """|sum_j l_j'(t) z_ij - h f(z_i(t), theta)| at each local time t of
    `points`, per element: array [N, len(points), n]."""
    z, theta = prob.split(np.asarray(x, dtype=np.float64))
    tau = prob.tab.tau
    out = np.zeros((prob.N, len(points), prob.n))
    for m, t in enumerate(points):
        lb = basis(tau, t)
        db = basis_derivative(tau, t)
        zt = np.einsum("j,ijs->is", lb, z)
        dz = np.einsum("j,ijs->is", db, z)
        out[:, m, :] = np.abs(dz - prob.h * prob.rhs(zt, theta, prob.escale))
    return out


def defect(prob: Problem, x):
    """Per-element defect (above) and its maximum."""
    tau = prob.tab.tau
    mids = [0.5 * (tau[m - 1] + tau[m]) for m in range(1, len(tau))]
    d = residual_at(prob, x, mids).max(axis=(1, 2))
    return d, float(d.max())


def interpolate(coarse: Problem, x, fine: Problem):
    """Fine-mesh x from the coarse solution x (above)."""
    zc, theta = coarse.split(np.asarray(x, dtype=np.float64))
    zf = np.zeros((fine.N, fine.K + 1, fine.n))
    for e in range(fine.N):
        c, i = divmod(e, fine.Nch)   # experimental condition, element within it
        for j in range(fine.K + 1):
            t = (i + fine.tab.tau[j]) * fine.h
            u = t / coarse.h
            ic = min(max(int(math.ceil(u)) - 1, 0), coarse.Nch - 1)
            zf[e, j] = basis(coarse.tab.tau, u - ic) @ zc[c * coarse.Nch + ic]
    return np.concatenate([zf.reshape(-1), theta])


@dataclasses.dataclass
class RefineResult:
    result: ipm.Result
    inst: object
    levels: int


def refine_solve(inst, theta0, opt: ipm.Options, defect_tol: float, max_levels: int,
                 max_elements: int = 0) -> RefineResult:
    res = ipm.solve(inst, theta0, opt)
    levels = 0
    for _ in range(max_levels):
        if res.status not in (ipm.SUCCESS, ipm.ACCEPTABLE):
            break
        prob = Problem(inst)
        _, dmax = defect(prob, res.x)
        nf = 2 * inst.N
        if not dmax > defect_tol or (max_elements and nf > max_elements):
            break
        fine_inst = inst.with_mesh(nf)
        xs = interpolate(prob, res.x, Problem(fine_inst))
        res = ipm.solve(fine_inst, xs[-inst.p:] if inst.p else None, opt, x_start=xs)
        inst = fine_inst
        levels += 1
    return RefineResult(res, inst, levels)
