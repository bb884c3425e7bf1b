"""Mesh refinement on the GPU (collo_defect, collo_interpolate, warm starts,
collo_refine_solve) against the oracle (paper Section "Static collocation
mesh limitations")."""
import numpy as np
import pytest

from paper_2607_12201_gb300 import workloads as W
from oracle import ipm as oipm, refine as orefine
from oracle.init import forward_sweep
from oracle.nlp import Problem as OProblem
from gpu_helpers import random_point

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def collo():
    from paper_2607_12201_gb300 import build
    build.build()
    from paper_2607_12201_gb300 import collo
    return collo


@pytest.mark.parametrize("make", [lambda: W.config1(), lambda: W.config2(N=100),
                                  lambda: W.small_network(n=3, r=5, N=7, seed=8)],
                         ids=["cascade_N50", "config2_N100", "tiny_N7"])
def test_defect_matches_oracle(collo, make):
    inst = make()
    oprob = OProblem(inst)
    for x in (random_point(oprob, 3)[0],
              np.concatenate([forward_sweep(oprob, inst.theta0)[0].reshape(-1), inst.theta0])):
        d_ref, m_ref = orefine.defect(oprob, x)
        with collo.Problem(inst) as prob:
            d, m = prob.defect(x)
        scale = max(1.0, m_ref)
        assert np.max(np.abs(d - d_ref)) <= 1e-12 * scale
        assert abs(m - m_ref) <= 1e-12 * scale


@pytest.mark.parametrize("Nc,Nf", [(50, 100), (50, 77), (7, 7), (40, 23)])
def test_interpolation_matches_oracle(collo, Nc, Nf):
    inst = W.config2(N=Nc)
    coarse, fine = OProblem(inst), OProblem(inst.with_mesh(Nf))
    x, _ = random_point(coarse, 5)
    ref = orefine.interpolate(coarse, x, fine)
    with collo.Problem(inst) as pc:
        with pc.refined(Nf) as pf:
            assert pf.N == Nf and pf.n_x == fine.n_x
            xf = collo.interpolate(pc, x, pf)
    # the two sides form the Lagrange basis in different orders
    assert np.max(np.abs(xf - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_warm_start_matches_oracle(collo, prec):
    """A solve from a given point (states and theta) instead of the forward sweep."""
    inst = W.config1().with_mesh(20)
    first = oipm.solve(inst.with_mesh(10), opt=oipm.Options(tol=1e-10))
    xs = orefine.interpolate(OProblem(inst.with_mesh(10)), first.x, OProblem(inst))
    ref = oipm.solve(inst, opt=oipm.Options(tol=1e-10), x_start=xs)
    P = collo.MIXED if prec == "mixed" else collo.FP64
    with collo.Problem(inst) as prob:
        prob.set_start(xs)
        res = prob.ipm_solve(precision=P, tol=1e-10, want_x=False)
    assert res["status"] == ref.status == 0
    assert res["iterations"] == ref.iterations
    assert np.max(np.abs(res["theta"] - ref.x[-2:]) / np.abs(ref.x[-2:])) <= 1e-8


def test_batched_refinement_matches_oracle(collo):
    """Three problems refined together: the cascade from N = 5 (refined twice,
    to N = 20), a small network from N = 6 and one whose defect is already
    below the tolerance; levels, final meshes and optima as the oracle's
    problem-by-problem loop."""
    insts = [W.config1().with_mesh(5),
             W.random_network(3, 5, n_obs=2, M=12, T=4.0, N=6, seed=8, theta0_spread=0.1),
             W.config1().with_mesh(200)]
    tol, levels_max = 2e-7, 2
    opt = oipm.Options(tol=1e-8)
    refs = [orefine.refine_solve(i, i.theta0, opt, tol, levels_max) for i in insts]
    probs = [collo.Problem(i) for i in insts]
    res, finals, levels = collo.refine_solve(probs, defect_tol=tol, max_levels=levels_max,
                                             precision=collo.FP64, tol=1e-8)
    for r, f, lv, ref in zip(res, finals, levels, refs):
        assert lv == ref.levels and f.N == ref.inst.N
        # solved on both sides; at the acceptable level (status 1) the two may
        # stop at different iterates inside the acceptable ball
        assert r["status"] in (0, 1) and ref.result.status in (0, 1)
        th = ref.result.x[-len(r["theta"]):]
        scale = np.abs(th) if not ref.inst.logscale else 1.0
        tol_th = 1e-6 if r["status"] == ref.result.status == 0 else 1e-4
        assert np.max(np.abs(r["theta"] - th) / scale) <= tol_th
    assert levels[0] == 2 and levels[2] == 0
    for f in finals:
        f.close()
    for p in probs:
        p.close()
