"""Several experimental conditions (paper Eq. 1d / 2e, lifted inputs of
Eq. 3) on the GPU against the oracle: evaluation, forward sweep, Newton step,
full solves, batches and mesh interpolation."""
import numpy as np
import pytest

from paper_2607_12201_gb300 import workloads as W
from oracle import ipm as oipm, refine as orefine
from oracle.init import forward_sweep
from oracle.nlp import Problem as OProblem
from gpu_helpers import assemble_J, assemble_W, newton_system, random_point, rel_max, sparse_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def collo():
    from paper_2607_12201_gb300 import build
    build.build()
    from paper_2607_12201_gb300 import collo
    return collo


CASES = {
    "c3_n6_N30": lambda: W.multi_condition(n=6, r=12, Nc=3, N=30, M=20, seed=1006),
    "c4_n10_N40": lambda: W.multi_condition(n=10, r=20, Nc=4, N=40, M=25, seed=1007),
    "c2_n14_N10": lambda: W.multi_condition(n=14, r=28, Nc=2, N=10, M=15, seed=1008),
}


@pytest.mark.parametrize("name", list(CASES))
def test_eval_matches_oracle(collo, name):
    inst = CASES[name]()
    oprob = OProblem(inst)
    x, lam = random_point(oprob, 11)
    ev = oprob.evaluate(x, lam, obj_factor=0.8)
    with collo.Problem(inst) as prob:
        assert prob.Nc == inst.Nc and prob.Nch == inst.N and prob.N == inst.Nc * inst.N
        out = prob.eval(x, lam, obj_factor=0.8)
    tol = 1e-13
    assert abs(out["phi"] - ev["phi"]) <= tol * max(1.0, abs(ev["phi"]))
    assert rel_max(out["c"], ev["c"]) <= tol
    assert rel_max(out["grad"], ev["grad"]) <= tol
    assert sparse_rel(assemble_J(oprob, out), ev["J"]) <= tol
    assert sparse_rel(assemble_W(oprob, out), ev["W"]) <= tol


@pytest.mark.parametrize("name", list(CASES))
def test_forward_sweep_matches_oracle(collo, name):
    inst = CASES[name]()
    oprob = OProblem(inst)
    z_ref, f_ref = forward_sweep(oprob, inst.theta0)
    with collo.Problem(inst) as prob:
        x, f = prob.initial_states(inst.theta0)
    assert f == f_ref
    z = x[:oprob.nz].reshape(z_ref.shape)
    assert np.max(np.abs(z - z_ref)) <= 1e-11 * max(1.0, np.max(np.abs(z_ref)))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_newton_step_matches_oracle(collo, name, prec):
    inst = CASES[name]()
    oprob = OProblem(inst)
    x, lam, zl, zu, _ = oipm.initial_point(oprob, inst.theta0, oipm.Options())
    mu, dw = 0.1, 1e-3
    dc = 1e-8 * mu ** 0.25
    ref = newton_system(oprob, x, lam, zl, zu, mu, dw, dc)
    P = collo.MIXED if prec == "mixed" else collo.FP64
    with collo.Problem(inst) as prob:
        prob.eval(x, lam)
        assert prob.kkt_factor(ref["sigma"], dw, dc, precision=P) == ref["inertia"]
        sol, info = prob.kkt_solve(ref["rhs"], refine_max=30, refine_tol=1e-14)
    err = np.linalg.norm(sol - ref["sol"]) / np.linalg.norm(ref["sol"])
    assert err <= 1e-10, (err, info)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_solve_matches_oracle(collo, prec):
    inst = CASES["c3_n6_N30"]()
    ref = oipm.solve(inst, opt=oipm.Options(tol=1e-8))
    P = collo.MIXED if prec == "mixed" else collo.FP64
    with collo.Problem(inst) as prob:
        res = prob.ipm_solve(precision=P, tol=1e-8, want_x=False)
    assert res["status"] == ref.status
    if ref.status in (0, 1):
        assert np.max(np.abs(10.0 ** (res["theta"] - ref.x[-inst.p:]) - 1.0)) <= 1e-6
        assert abs(res["phi"] - ref.phi) <= 1e-6 * abs(ref.phi)
    else:
        assert res["iterations"] == ref.iterations


def test_conditions_in_a_batch_equal_alone_bitwise(collo):
    insts = [CASES["c3_n6_N30"](), W.config2(N=60), CASES["c2_n14_N10"]()]
    alone = []
    for inst in insts:
        with collo.Problem(inst) as pb:
            alone.append(pb.ipm_solve(precision=collo.MIXED, want_x=False, max_iter=10))
    probs = [collo.Problem(i) for i in insts]
    mixed = collo.batch_solve(probs, precision=collo.MIXED, max_iter=10)
    for a, b in zip(alone, mixed):
        assert a["iterations"] == b["iterations"]
        assert np.array_equal(a["theta"], b["theta"])
    for pb in probs:
        pb.close()


def test_interpolation_and_defect_with_conditions(collo):
    inst = CASES["c3_n6_N30"]()
    coarse, fine = OProblem(inst), OProblem(inst.with_mesh(45))
    x, _ = random_point(coarse, 5)
    ref = orefine.interpolate(coarse, x, fine)
    d_ref, m_ref = orefine.defect(coarse, x)
    with collo.Problem(inst) as pc:
        d, m = pc.defect(x)
        with pc.refined(45) as pf:
            assert pf.Nc == inst.Nc and pf.Nch == 45
            xf = collo.interpolate(pc, x, pf)
    # the two sides form the Lagrange basis in different orders
    assert np.max(np.abs(xf - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(d - d_ref)) <= 1e-12 * max(1.0, m_ref)
