"""Lifted (relaxed-equality) condensed-space Newton step on the GPU against the
oracle (``oracle.lifted``; paper Section "Optimization framework
configurations": the LiftedKKT form).

The GPU factors Kc = W + Sigma_x + dw I + J^T (Sigma_s + dw) J by Cholesky in
its own order (element interiors, block cyclic reduction over the chain of
first points, parameter block) and refines against the unreduced system; the
oracle factors the same matrix in natural block order.  Cases cover element
blocks in shared memory and in global memory (40 and 80 species), parameter
blocks in shared and global memory, a single element, Gauss-Legendre K = 4 and
chains cut at experimental conditions."""
import dataclasses

import numpy as np
import pytest

from paper_2607_12201_gb300 import workloads as W
from oracle import lifted
from oracle.nlp import Problem as OProblem

pytestmark = pytest.mark.gpu


def gauss(inst):
    return dataclasses.replace(inst, K=4, scheme="gauss")


CASES = {
    "cascade_N50": lambda: W.config1(),
    "tiny_N1": lambda: W.small_network(n=3, r=4, N=1, seed=7),
    "tiny_N7": lambda: W.small_network(n=3, r=5, N=7, seed=8),
    "one_species_N3": lambda: W.random_network(1, 2, n_obs=1, M=5, T=2.0, N=3, seed=9),
    "config2_N400": lambda: W.config2(),
    "n13_N20": lambda: W.random_network(13, 26, n_obs=4, M=20, T=5.0, N=20, seed=52,
                                        theta0_spread=0.1),
    # element block of 90 + 60 + 30 = 180 unknowns: global-memory path
    "config3_N40": lambda: W.config3(N=40),
    "gauss_cascade_N50": lambda: gauss(W.config1()),
    "gauss_n13_N20": lambda: gauss(W.random_network(13, 26, n_obs=4, M=20, T=5.0, N=20, seed=52,
                                                    theta0_spread=0.1)),
    "conditions_3x30": lambda: W.multi_condition(),
    # element blocks of 280 and 560 unknowns (factored in global memory); the
    # second has p = 160, so its parameter block is factored in global memory too
    "n40_N6": lambda: W.random_network(40, 80, n_obs=8, M=40, T=5.0, N=6, seed=61,
                                       theta0_spread=0.1),
    "n80_N4": lambda: W.random_network(80, 160, n_obs=8, M=40, T=5.0, N=4, seed=62,
                                       theta0_spread=0.1),
}


@pytest.fixture(scope="module")
def collo():
    from paper_2607_12201_gb300 import build
    build.build()
    from paper_2607_12201_gb300 import collo
    return collo


def _state(oprob, opt, seed, lam_scale=0.3):
    rng = np.random.default_rng(seed)
    inst = oprob.inst
    x = rng.uniform(0.2, 1.2, oprob.n_x)
    lo, hi = inst.theta_lo, inst.theta_hi
    x[oprob.nz:] = lo + (hi - lo) * rng.uniform(0.3, 0.7, oprob.p)
    if inst.logscale:
        x[oprob.nz:] = rng.uniform(-1.0, 0.5, oprob.p)
    m = oprob.n_c
    r = opt.r()
    return lifted.State(x=x, s=r * rng.uniform(-0.9, 0.9, m),
                        lam=lam_scale * rng.standard_normal(m),
                        zl=rng.uniform(0.5, 2.0, oprob.p), zu=rng.uniform(0.5, 2.0, oprob.p),
                        vl=rng.uniform(0.5, 2.0, m), vu=rng.uniform(0.5, 2.0, m))


def _gpu_step(collo, inst, st, ref, dw, refine_max=20):
    with collo.Problem(inst) as prob:
        prob.eval(st.x, st.lam)
        pd = prob.lifted_factor(ref["sigma_x"], ref["sigma_s"], dw)
        assert pd
        dx, ds, dl, info = prob.lifted_solve(ref["r_x"], ref["r_s"], ref["r_c"],
                                             refine_max=refine_max, refine_tol=1e-13)
    return dx, ds, dl, info


def _backward(M, sol, b):
    r = b - M @ sol
    return float(np.max(np.abs(r)) / max(1.0, np.max(np.abs(b))))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _forward_tol(ref, n_x):
    """Ten times the oracle's own distance from a sparse LU solve (scipy's
    splu, refined) of the unreduced system, at least 1e-9: the random and
    start iterates reach condition numbers where two backward-stable FP64
    solves legitimately differ in the 7th digit."""
    import scipy.sparse.linalg as spla
    b = np.concatenate([ref["r_x"], ref["r_s"], ref["r_c"]])
    lu = spla.splu(ref["M"].tocsc())
    ex = lu.solve(b)
    for _ in range(3):
        ex = ex + lu.solve(b - ref["M"] @ ex)
    m = ref["r_s"].size
    spread = max(_rel(ref["dx"], ex[:n_x]), _rel(ref["ds"], ex[n_x:n_x + m]),
                 _rel(ref["dlam"], ex[n_x + m:]))
    return max(1e-9, 10.0 * spread)


@pytest.mark.parametrize("name", [c for c in CASES if c != "n80_N4"])
@pytest.mark.parametrize("dw", [0.0, 1e-2])
def test_lifted_step_matches_oracle(collo, name, dw):
    """Relaxation r = 1e-4 at a random iterate: backward error of the GPU step
    on the unreduced system <= 1e-13, forward agreement with the oracle within
    the conditioning-derived tolerance."""
    inst = CASES[name]()
    oprob = OProblem(inst)
    opt = lifted.Options(relax=1e-4)
    st = _state(oprob, opt, 21)
    ev = oprob.evaluate(st.x, st.lam)
    try:
        ref = lifted.newton_direction(oprob, ev, st, 0.05, dw, opt)
    except lifted.NotPositiveDefinite:
        pytest.skip("not positive definite at this point")
    dx, ds, dl, info = _gpu_step(collo, inst, st, ref, dw)
    b = np.concatenate([ref["r_x"], ref["r_s"], ref["r_c"]])
    assert _backward(ref["M"], np.concatenate([dx, ds, dl]), b) <= 1e-13, info
    tol = _forward_tol(ref, oprob.n_x)
    assert _rel(dx, ref["dx"]) <= tol
    assert _rel(ds, ref["ds"]) <= tol
    assert _rel(dl, ref["dlam"]) <= tol


@pytest.mark.parametrize("dw", [0.1, 10.0])
def test_lifted_step_with_parameter_block_in_global_memory(collo, dw):
    """80 species, p = 160: element blocks of 560 unknowns and a 160 x 160
    parameter block, both factored in global memory; small multipliers keep
    the condensed matrix positive definite."""
    inst = CASES["n80_N4"]()
    oprob = OProblem(inst)
    opt = lifted.Options(relax=1e-4)
    st = _state(oprob, opt, 21, lam_scale=0.05)
    ev = oprob.evaluate(st.x, st.lam)
    ref = lifted.newton_direction(oprob, ev, st, 0.05, dw, opt)
    dx, ds, dl, info = _gpu_step(collo, inst, st, ref, dw)
    b = np.concatenate([ref["r_x"], ref["r_s"], ref["r_c"]])
    assert _backward(ref["M"], np.concatenate([dx, ds, dl]), b) <= 1e-13, info
    tol = _forward_tol(ref, oprob.n_x)
    assert _rel(dx, ref["dx"]) <= tol
    assert _rel(ds, ref["ds"]) <= tol
    assert _rel(dl, ref["dlam"]) <= tol


@pytest.mark.parametrize("name", ["cascade_N50", "config2_N400", "n13_N20", "config3_N40",
                                  "gauss_cascade_N50", "conditions_3x30"])
def test_lifted_step_at_ipm_start_matches_oracle(collo, name):
    """The interior-point start with the default relaxation r = 1e-8: slacks
    near 0 with unit bound duals, Sigma_s about 2 / r."""
    inst = CASES[name]()
    oprob = OProblem(inst)
    opt = lifted.Options()
    st, _ = lifted.initial_point(oprob, inst.theta0, opt)
    ev = oprob.evaluate(st.x, st.lam)
    dw = 0.0
    try:
        ref = lifted.newton_direction(oprob, ev, st, opt.mu_init, dw, opt)
    except lifted.NotPositiveDefinite:
        dw = 1e-4
        ref = lifted.newton_direction(oprob, ev, st, opt.mu_init, dw, opt)
    dx, ds, dl, info = _gpu_step(collo, inst, st, ref, dw)
    b = np.concatenate([ref["r_x"], ref["r_s"], ref["r_c"]])
    assert _backward(ref["M"], np.concatenate([dx, ds, dl]), b) <= 1e-12, info
    tol = _forward_tol(ref, oprob.n_x)
    assert _rel(dx, ref["dx"]) <= tol
    assert _rel(ds, ref["ds"]) <= tol
    assert _rel(dl, ref["dlam"]) <= tol


@pytest.mark.parametrize("seed", [1, 2, 5, 8])
def test_lifted_positive_definiteness_matches_oracle(collo, seed):
    """Large multipliers make W indefinite; the GPU's Cholesky fails exactly
    where the oracle's does across a sweep of dw."""
    inst = W.small_network(n=2, r=3, N=3, seed=17)
    oprob = OProblem(inst)
    opt = lifted.Options(relax=1e-3)
    st = _state(oprob, opt, seed, lam_scale=30.0)
    ev = oprob.evaluate(st.x, st.lam)
    sx, ss = lifted.sigmas(oprob, st, opt.r())
    seen = set()
    with collo.Problem(inst) as prob:
        prob.eval(st.x, st.lam)
        for dw in [0.0, 1e-3, 1e-1, 1.0, 10.0, 100.0, 1e3, 1e4]:
            Kc = lifted.condensed_matrix(ev["J"], ev["W"], sx, ss, dw)
            try:
                lifted.DenseCholesky(Kc)
                ok = True
            except lifted.NotPositiveDefinite:
                ok = False
            assert prob.lifted_factor(sx, ss, dw) == ok, dw
            seen.add(ok)
    assert seen == {True, False}


def test_lifted_solve_needs_a_current_positive_definite_factorization(collo):
    inst = CASES["tiny_N7"]()
    oprob = OProblem(inst)
    opt = lifted.Options(relax=1e-3)
    st = _state(oprob, opt, 3)
    sx, ss = lifted.sigmas(oprob, st, opt.r())
    zx, zc = np.zeros(oprob.n_x), np.zeros(oprob.n_c)
    with collo.Problem(inst) as prob:
        with pytest.raises(collo.ColloError) as e:
            prob.lifted_factor(sx, ss, 0.0)
        assert e.value.status == collo.ERR_NOT_EVALUATED
        prob.eval(st.x, st.lam)
        with pytest.raises(collo.ColloError) as e:
            prob.lifted_solve(zx, zc, zc)
        assert e.value.status == collo.ERR_NOT_FACTORED
        assert prob.lifted_factor(sx, ss, 1e4)
        dx, ds, dl, _ = prob.lifted_solve(zx, zc, zc)
        assert not np.any(dx) and not np.any(ds) and not np.any(dl)
        prob.eval(st.x, st.lam)           # a new evaluation invalidates the factor
        with pytest.raises(collo.ColloError) as e:
            prob.lifted_solve(zx, zc, zc)
        assert e.value.status == collo.ERR_NOT_FACTORED
        with pytest.raises(collo.ColloError) as e:
            prob.lifted_factor(sx, ss, -1.0)
        assert e.value.status == collo.ERR_INVALID_ARG


def _lifted_compare(res, ref, inst, th_tol=1e-6):
    assert res["status"] == ref.status
    th_ref = ref.x[-inst.p:]
    rel = np.max(np.abs(res["theta"] - th_ref) / np.maximum(np.abs(th_ref), 1e-12))
    assert rel <= th_tol, (res["theta"], th_ref)
    assert abs(res["phi"] - ref.phi) <= th_tol * max(1.0, abs(ref.phi))


@pytest.mark.parametrize("name", ["cascade_N50", "gauss_cascade_N50"])
def test_lifted_ipm_solve_matches_oracle(collo, name):
    """The whole relaxed-equality interior-point solve (r = 1e-8) against the
    oracle's on the well-identified cascade: status, iteration count, theta
    and Phi."""
    inst = CASES[name]()
    ref = lifted.solve(inst)
    with collo.Problem(inst) as prob:
        res = prob.lifted_ipm_solve()
    _lifted_compare(res, ref, inst)
    assert res["iterations"] == ref.iterations


def test_lifted_ipm_solve_on_a_network_reaches_the_oracle_objective(collo):
    """A 4-species network whose sixth parameter is not identified (the
    oracle's solve leaves it anywhere between -4.86 and -5.0, its bound,
    depending on the tolerance): the lifted steps carry the forward error of
    a matrix with Sigma_s near mu / r^2, so the two trajectories separate along
    that direction.  Status and the objective must agree."""
    inst = W.random_network(4, 8, n_obs=3, M=20, T=5.0, N=40, seed=41, theta0_spread=0.1)
    ref = lifted.solve(inst)
    with collo.Problem(inst) as prob:
        res = prob.lifted_ipm_solve()
    assert res["status"] == ref.status
    assert abs(res["phi"] - ref.phi) <= 1e-5 * abs(ref.phi)


def test_lifted_ipm_solve_status_on_config2_matches_oracle(collo):
    """Config 2 from its theta0: the oracle's lifted solve ends in a line-search
    failure; the GPU's ends with the same status and follows the oracle's
    trajectory through the first iterations."""
    inst = CASES["config2_N400"]()
    hist = []
    ref = lifted.solve(inst, on_iter=hist.append)
    with collo.Problem(inst) as prob:
        res = prob.lifted_ipm_solve()
        k = max(1, len(hist) // 4)
        early = prob.lifted_ipm_solve(max_iter=k)
    assert res["status"] == ref.status
    th_ref = hist[k - 1]["theta"]
    rel = np.max(np.abs(early["theta"] - th_ref) / np.maximum(np.abs(th_ref), 1e-12))
    assert rel <= 1e-6, rel


def test_lifted_ipm_solve_with_experimental_conditions(collo):
    """Three experimental conditions (chains cut at each condition's first
    element, theta shared): status, objective and theta within the
    tolerance's ball (the oracle's own theta moves by 2e-5 between tolerances
    1e-6 and 1e-8 here), iteration count within two."""
    inst = CASES["conditions_3x30"]()
    ref = lifted.solve(inst)
    with collo.Problem(inst) as prob:
        res = prob.lifted_ipm_solve()
    assert res["status"] == ref.status
    assert abs(res["phi"] - ref.phi) <= 1e-6 * abs(ref.phi)
    th_ref = ref.x[-inst.p:]
    assert np.max(np.abs(res["theta"] - th_ref) / np.abs(th_ref)) <= 1e-4
    assert abs(res["iterations"] - ref.iterations) <= 2
