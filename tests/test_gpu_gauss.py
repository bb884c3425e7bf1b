"""Gauss-Legendre collocation with K = 4 (the paper's node choice, section
"Collocation equation with condition independence"; K = 4 in "Optimization
framework configurations") on the GPU against the oracle's scheme="gauss".

Continuity goes through the extrapolated end value sum_j b_j z_ij, b_j = l_j(1)
(Eq. 2c), so the element block holds the outgoing continuity row and the
chain block of element i is (z_i0, c_i0).  Cases cover the register-tile
element path (10n + p <= 124), the shared-memory and global-slab large-element
paths, several experimental conditions (chains cut at each condition's first
element) and mixed batches of Gauss and Radau problems."""
import dataclasses

import numpy as np
import pytest

from paper_2607_12201_gb300 import workloads as W
from oracle import ipm as oipm
from oracle.init import forward_sweep
from oracle.nlp import Problem as OProblem
from gpu_helpers import (assemble_J, assemble_W, newton_system, random_point, rel_max,
                         sparse_rel)

pytestmark = pytest.mark.gpu


def gauss(inst):
    return dataclasses.replace(inst, K=4, scheme="gauss")


CASES = {
    "cascade_N50": lambda: gauss(W.config1()),
    "tiny_N1": lambda: gauss(W.small_network(n=3, r=4, N=1, seed=7)),
    "tiny_N2": lambda: gauss(W.small_network(n=2, r=3, N=2, seed=17)),
    "tiny_N7": lambda: gauss(W.small_network(n=3, r=5, N=7, seed=8)),
    "one_species_N3": lambda: gauss(W.random_network(1, 2, n_obs=1, M=5, T=2.0, N=3, seed=9)),
    "n4_N33": lambda: gauss(W.random_network(4, 8, n_obs=2, M=20, T=5.0, N=33, seed=19)),
    # 10n + p = 120 rows: the largest register-tiled element block
    "config2_N400": lambda: gauss(W.config2()),
    # 10n + p = 156 rows (shared memory) and, in FP64, 180 rows (global slab)
    "n13_N20": lambda: gauss(W.random_network(13, 26, n_obs=4, M=20, T=5.0, N=20, seed=52,
                                              theta0_spread=0.1)),
    "n15_N9": lambda: gauss(W.random_network(15, 30, n_obs=4, M=20, T=5.0, N=9, seed=53,
                                             theta0_spread=0.1)),
    # three experimental conditions of 30 elements: chains cut at 30 and 60
    "conditions_3x30": lambda: gauss(W.multi_condition()),
}


@pytest.fixture(scope="module")
def collo():
    from paper_2607_12201_gb300 import build
    build.build()
    from paper_2607_12201_gb300 import collo
    return collo


def _point(oprob, seed):
    x, lam = random_point(oprob, seed, lam_scale=0.3)
    rng = np.random.default_rng(seed + 1)
    zl = rng.uniform(0.5, 2.0, oprob.p)
    zu = rng.uniform(0.5, 2.0, oprob.p)
    return x, lam, zl, zu


def backward_error(K, x, b):
    r = b - K @ x
    Kinf = abs(K).sum(axis=1).max()
    return float(np.max(np.abs(r)) / (Kinf * np.max(np.abs(x)) + np.max(np.abs(b))))


def test_sizes_report_gauss_layout(collo):
    inst = CASES["tiny_N7"]()
    with collo.Problem(inst) as prob:
        assert prob.sizes.K == 4
        assert prob.n_x == inst.n * inst.N * 5 + inst.p
        assert prob.n_c == inst.n * inst.N * 5


@pytest.mark.parametrize("name", ["cascade_N50", "tiny_N1", "tiny_N7", "one_species_N3",
                                  "config2_N400", "n13_N20", "conditions_3x30"])
def test_gauss_eval_matches_oracle(collo, name):
    inst = CASES[name]()
    oprob = OProblem(inst)
    x, lam = random_point(oprob, 11)
    ev = oprob.evaluate(x, lam, obj_factor=0.8)
    with collo.Problem(inst) as prob:
        out = prob.eval(x, lam, obj_factor=0.8)
    tol = 1e-13
    assert abs(out["phi"] - ev["phi"]) <= tol * max(1.0, abs(ev["phi"]))
    assert rel_max(out["c"], ev["c"]) <= tol
    assert rel_max(out["grad"], ev["grad"]) <= tol
    assert sparse_rel(assemble_J(oprob, out), ev["J"]) <= tol
    assert sparse_rel(assemble_W(oprob, out), ev["W"]) <= tol


@pytest.mark.parametrize("name", ["cascade_N50", "tiny_N7", "config2_N400", "n13_N20",
                                  "conditions_3x30"])
def test_gauss_forward_sweep_matches_oracle(collo, name):
    """4n <= 32 runs the one-warp chord sweep, larger systems the CTA sweep."""
    inst = CASES[name]()
    oprob = OProblem(inst)
    th = np.array(inst.theta0, dtype=float)
    z_ref, f_ref = forward_sweep(oprob, th)
    with collo.Problem(inst) as prob:
        x, f = prob.initial_states(th)
    assert f == f_ref
    z = x[:oprob.nz].reshape(z_ref.shape)
    assert np.max(np.abs(z - z_ref)) <= 1e-11 * max(1.0, np.max(np.abs(z_ref)))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("dw", [0.0, 1e-2])
def test_gauss_newton_step_matches_oracle_fp64(collo, name, dw):
    inst = CASES[name]()
    oprob = OProblem(inst)
    x, lam, zl, zu = _point(oprob, 21)
    mu = 0.05
    dc = 1e-8 * mu ** 0.25
    ref = newton_system(oprob, x, lam, zl, zu, mu, dw, dc)
    with collo.Problem(inst) as prob:
        prob.eval(x, lam)
        inertia = prob.kkt_factor(ref["sigma"], dw, dc, precision=collo.FP64)
        assert inertia == ref["inertia"]
        sol, info = prob.kkt_solve(ref["rhs"], refine_max=3, refine_tol=1e-14)
    err = np.linalg.norm(sol - ref["sol"]) / np.linalg.norm(ref["sol"])
    assert backward_error(ref["K"], sol, ref["rhs"]) <= 1e-15
    assert err <= 1e-10, (err, info)


@pytest.mark.parametrize("name", ["cascade_N50", "n4_N33", "config2_N400", "n13_N20",
                                  "n15_N9", "conditions_3x30"])
def test_gauss_newton_step_at_ipm_start_mixed_precision(collo, name):
    """FP32 factorization + FP64 refinement reaches the oracle's FP64 step."""
    inst = CASES[name]()
    oprob = OProblem(inst)
    opt = oipm.Options()
    x, lam, zl, zu, _ = oipm.initial_point(oprob, inst.theta0, opt)
    mu = 0.1
    dc = 1e-8 * mu ** 0.25
    dw = 1e-3
    ref = newton_system(oprob, x, lam, zl, zu, mu, dw, dc)
    with collo.Problem(inst) as prob:
        prob.eval(x, lam)
        inertia = prob.kkt_factor(ref["sigma"], dw, dc, precision=collo.MIXED)
        assert inertia == ref["inertia"]
        sol, info = prob.kkt_solve(ref["rhs"], refine_max=30, refine_tol=1e-14)
    err = np.linalg.norm(sol - ref["sol"]) / np.linalg.norm(ref["sol"])
    assert err <= 1e-10, (err, info)


def _compare(res, ref, inst):
    assert res["status"] == ref.status
    th_ref = ref.x[-inst.p:]
    rel = np.max(np.abs(res["theta"] - th_ref) / np.maximum(np.abs(th_ref), 1e-12))
    assert rel <= 1e-6, (res["theta"], th_ref)
    assert abs(res["phi"] - ref.phi) <= 1e-6 * max(1.0, abs(ref.phi))


def test_gauss_cascade_solve_matches_oracle(collo):
    inst = CASES["cascade_N50"]()
    ref = oipm.solve(inst)
    with collo.Problem(inst) as prob:
        res = prob.ipm_solve()
    _compare(res, ref, inst)
    assert res["iterations"] == ref.iterations


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["small_n4_N40", "n13_N20", "conditions_3x30"])
def test_gauss_network_solves_match_oracle(collo, name, prec):
    inst = (gauss(W.random_network(4, 8, n_obs=3, M=20, T=5.0, N=40, seed=41,
                                   theta0_spread=0.1))
            if name == "small_n4_N40" else CASES[name]())
    ref = oipm.solve(inst)
    with collo.Problem(inst) as prob:
        res = prob.ipm_solve(precision=collo.MIXED if prec == "mixed" else collo.FP64)
    _compare(res, ref, inst)


def test_gauss_config2_solve_matches_oracle(collo):
    inst = CASES["config2_N400"]()
    ref = oipm.solve(inst)
    with collo.Problem(inst) as prob:
        r64 = prob.ipm_solve(precision=collo.FP64)
        rmx = prob.ipm_solve(precision=collo.MIXED)
    _compare(r64, ref, inst)
    _compare(rmx, ref, inst)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_gauss_and_radau_in_one_batch_equal_alone(collo, prec):
    """Each problem's iterates are the same alone and in a batch that mixes
    both schemes and all three element paths."""
    P = collo.MIXED if prec == "mixed" else collo.FP64
    insts = [CASES["n4_N33"](), W.random_network(4, 8, n_obs=2, M=20, T=5.0, N=33, seed=19),
             CASES["n13_N20"](), CASES["n15_N9"](), CASES["conditions_3x30"]()]
    alone = []
    for inst in insts:
        with collo.Problem(inst) as pb:
            alone.append(pb.ipm_solve(precision=P, want_x=True, max_iter=10))
    probs = [collo.Problem(inst) for inst in insts]
    mixed = collo.batch_solve(probs, precision=P, max_iter=10, want_x=True)
    for a, b in zip(alone, mixed):
        assert a["status"] == b["status"]
        assert a["iterations"] == b["iterations"]
        assert np.array_equal(a["theta"], b["theta"])
        assert np.array_equal(a["x"], b["x"])
    for pb in probs:
        pb.close()


def test_gauss_refinement_defect_and_interpolation_match_oracle(collo):
    from oracle import refine as orefine
    inst = CASES["tiny_N7"]()
    coarse, fine = OProblem(inst), OProblem(inst.with_mesh(17))
    x, _ = random_point(coarse, 5)
    ref = orefine.interpolate(coarse, x, fine)
    d_ref, m_ref = orefine.defect(coarse, x)
    with collo.Problem(inst) as pc:
        d, m = pc.defect(x)
        with pc.refined(17) as pf:
            assert pf.sizes.K == 4 and pf.n_x == fine.n_x
            xf = collo.interpolate(pc, x, pf)
    assert np.max(np.abs(xf - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
    scale = max(1.0, m_ref)
    assert np.max(np.abs(d - d_ref)) <= 1e-12 * scale
    assert abs(m - m_ref) <= 1e-12 * scale
