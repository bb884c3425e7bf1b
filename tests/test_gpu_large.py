"""Parity at the stated sizes of the large workloads: the stiff network at
N = 2000 (evaluation, FP64 Newton step, full FP64 and mixed solves), the
multistart-batch and serving-stream shapes at their largest species counts,
and an uneven batch, each against the CPU oracle.

The oracle's solves of these instances take minutes to hours on a CPU; their
optima are stored in tests/golden/oracle_optima_large.json by
tests/golden/make_large_oracle_optima.py (oracle only).  Evaluations and
Newton steps are recomputed by the oracle here.
"""
import json
import os

import numpy as np
import pytest

from paper_2607_12201_gb300 import workloads as W
from oracle.nlp import Problem as OProblem
from gpu_helpers import assemble_J, assemble_W, newton_system, random_point, sparse_rel

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "oracle_optima_large.json")


@pytest.fixture(scope="module")
def collo():
    from paper_2607_12201_gb300 import build
    build.build()
    from paper_2607_12201_gb300 import collo
    return collo


@pytest.fixture(scope="module")
def config3():
    return W.config3()


def golden(name):
    if not os.path.exists(GOLDEN):
        pytest.skip("no stored oracle optima")
    data = json.load(open(GOLDEN))
    if name not in data:
        pytest.skip(f"no stored oracle optimum for {name}")
    return data[name]


def test_config3_full_size_evaluation_matches_oracle(collo, config3):
    """Residuals, Jacobian and Hessian on all 2000 x 3 (element, node) pairs."""
    oprob = OProblem(config3)
    x, lam = random_point(oprob, 7, lam_scale=0.5)
    ev = oprob.evaluate(x, lam, 0.8)
    with collo.Problem(config3) as prob:
        out = prob.eval(x, lam, obj_factor=0.8)
    scale = max(1.0, np.max(np.abs(ev["c"])))
    assert np.max(np.abs(out["c"] - ev["c"])) / scale <= 1e-13
    assert abs(out["phi"] - ev["phi"]) <= 1e-13 * max(1.0, abs(ev["phi"]))
    gscale = max(1.0, np.max(np.abs(ev["grad"])))
    assert np.max(np.abs(out["grad"] - ev["grad"])) / gscale <= 1e-13
    assert sparse_rel(assemble_J(oprob, out), ev["J"]) <= 1e-13
    assert sparse_rel(assemble_W(oprob, out), ev["W"]) <= 1e-13


def backward_error(K, x, b):
    r = b - K @ x
    Kinf = abs(K).sum(axis=1).max()
    return float(np.max(np.abs(r)) / (Kinf * np.max(np.abs(x)) + np.max(np.abs(b))))


def test_config3_full_size_newton_step_matches_oracle(collo, config3):
    """The FP64 Newton step at N = 2000 (11 cyclic-reduction levels) against the
    oracle's natural-order block elimination of the same system: backward error
    at the rounding level, forward agreement 1e-9 (the tolerance of the stiff
    network, whose KKT condition number is near 1e24).  The mixed path's
    refinement either reaches the same step or reports a residual above the
    escalation threshold (1e-6), which sends the interior-point method to FP64."""
    oprob = OProblem(config3)
    x, lam = random_point(oprob, 21, lam_scale=0.3)
    rng = np.random.default_rng(22)
    zl = rng.uniform(0.5, 2.0, oprob.p)
    zu = rng.uniform(0.5, 2.0, oprob.p)
    mu, dw = 0.05, 1e-2
    dc = 1e-8 * mu ** 0.25
    ref = newton_system(oprob, x, lam, zl, zu, mu, dw, dc)
    with collo.Problem(config3) as prob:
        prob.eval(x, lam)
        prob.kkt_factor(ref["sigma"], dw, dc, precision=collo.FP64)
        sol, info = prob.kkt_solve(ref["rhs"], refine_max=3, refine_tol=1e-14)
        prob.kkt_factor(ref["sigma"], dw, dc, precision=collo.MIXED)
        solm, infom = prob.kkt_solve(ref["rhs"], refine_max=10, refine_tol=1e-10)
    assert backward_error(ref["K"], sol, ref["rhs"]) <= 1e-15
    err = np.linalg.norm(sol - ref["sol"]) / np.linalg.norm(ref["sol"])
    assert err <= 1e-9, (err, info)
    if infom["residual"] <= 1e-10:
        errm = np.linalg.norm(solm - ref["sol"]) / np.linalg.norm(ref["sol"])
        assert errm <= 1e-8, (errm, infom)
    else:
        assert infom["residual"] > 1e-6, infom


def _theta_rel(a, b):
    """max |k_a / k_b - 1| over the rate constants k = 10^theta."""
    return float(np.max(np.abs(10.0 ** (np.asarray(a) - np.asarray(b)) - 1.0)))


def _compare_optimum(res, ref):
    """A converged solve: same status, rate constants within 1e-6 relative, Phi
    within 1e-6.  A failed one (line-search failure, the paper's "R"): the same
    status; its trajectory is compared at checkpoints (below)."""
    assert res["status"] == ref["status"], (res["status"], ref["status"])
    if ref["status"] in (0, 1):
        assert _theta_rel(res["theta"], ref["theta"]) <= 1e-6
        assert abs(res["phi"] - ref["phi"]) <= 1e-6 * abs(ref["phi"])


# A failed solve (line-search failure, the paper's "R": no restoration phase)
# ends after a stretch of steps near alpha_min, where rounding decides ties in
# the filter tests, so its final point is not a parity target.  Its trajectory
# is: the library's iterate after m Newton steps (max_iter = m) against the
# oracle's.  In FP64 the rate constants k = 10^theta agree within 1e-6 over the
# first quarter of the solve (measured: 1e-12 to 8e-8); later the iterates
# wander on a nearly singular barrier problem and the two drift apart (1e-6 to
# 2e-5 by the middle), which is printed, not asserted.  The mixed path takes
# its inertia from FP32 pivots, which at such iterates may choose another
# regularisation and leave the trajectory early: for it only the status is a
# parity target, and the divergence is printed.
def _checkpoints(ref):
    n = ref["iterations"]
    return sorted({max(1, n // 4), max(1, n // 2), max(1, (3 * n) // 4), max(1, n - 5)})


def _compare_trajectory(run, ref, asserted, first_tol=1e-6):
    """run(max_iter) -> result dict."""
    first = max(1, ref["iterations"] // 4)
    for m in _checkpoints(ref):
        res = run(m)
        if not asserted:   # the mixed path may fail before the checkpoint
            rel = _theta_rel(res["theta"], ref["trajectory"][m - 1])
            print(f"checkpoint {m}/{ref['iterations']}: {rel:.2e} (status {res['status']})")
            continue
        assert res["status"] == -5 and res["iterations"] == m
        rel = _theta_rel(res["theta"], ref["trajectory"][m - 1])
        print(f"checkpoint {m}/{ref['iterations']}: {rel:.2e}")
        if m == first:
            assert rel <= first_tol, (m, rel)


def _solve_and_compare(collo, inst, ref, P, first_tol=1e-6):
    with collo.Problem(inst) as prob:
        res = prob.ipm_solve(precision=P, tol=ref["tol"], want_x=False)
        _compare_optimum(res, ref)
        if "trajectory" in ref:
            _compare_trajectory(lambda m: prob.ipm_solve(precision=P, tol=ref["tol"],
                                                         want_x=False, max_iter=m), ref,
                                asserted=P == collo.FP64, first_tol=first_tol)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_config3_full_size_solve_matches_oracle(collo, config3, prec):
    ref = golden("config3_N2000")
    P = collo.MIXED if prec == "mixed" else collo.FP64
    # the stiff network's KKT systems have condition numbers near 1e24: two
    # backward-stable FP64 steps agree to 1e-9 only, and the trajectories are
    # 2.5e-5 apart after a quarter of the (failing) solve
    _solve_and_compare(collo, config3, ref, P, first_tol=1e-4)


@pytest.mark.parametrize("name,make", [
    ("config4_n50_N100", lambda: W.random_network(50, 100, log10k=(-2.0, 1.0), n_obs=4, M=50,
                                                  T=20.0, N=100, seed=4001, theta0_spread=0.1)),
    ("config5_n100_N40", lambda: W.random_network(100, 200, log10k=(-2.0, 1.0), n_obs=4, M=50,
                                                  T=20.0, N=40, seed=5001, theta0_spread=0.1)),
])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_largest_species_counts_solve_matches_oracle(collo, name, make, prec):
    """n = 50 (element blocks of 500 rows, p = 100) and n = 100 (1000 rows,
    p = 200: the parameter Schur block in global memory)."""
    ref = golden(name)
    inst = make()
    P = collo.MIXED if prec == "mixed" else collo.FP64
    _solve_and_compare(collo, inst, ref, P)


BATCH = [(5, 160, 6001), (9, 90, 6002), (14, 120, 6003), (22, 60, 6004), (31, 45, 6005),
         (40, 30, 6006)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_uneven_batch_matches_per_instance_oracle(collo, prec):
    """Six networks of 5 to 40 species (element blocks of 50 to 400 rows: register
    tiles, shared memory and global slabs in one batch) solved together; each
    result against the oracle's solve of that instance alone."""
    refs = [golden(f"batch_n{n}_N{N}") for n, N, _ in BATCH]
    insts = [W.random_network(n, 2 * n, log10k=(-2.0, 1.0), n_obs=min(4, n), M=50, T=20.0,
                              N=N, seed=s, theta0_spread=0.1) for n, N, s in BATCH]
    P = collo.MIXED if prec == "mixed" else collo.FP64
    probs = [collo.Problem(i) for i in insts]
    res = collo.batch_solve(probs, precision=P, tol=refs[0]["tol"])
    for r, ref in zip(res, refs):
        _compare_optimum(r, ref)
    # failed members: their trajectories, each in a batch of its own
    for k, ref in enumerate(refs):
        if "trajectory" in ref:
            _compare_trajectory(lambda m: collo.batch_solve([probs[k]], precision=P,
                                                            tol=ref["tol"], max_iter=m)[0], ref,
                                asserted=P == collo.FP64)
    for pb in probs:
        pb.close()
