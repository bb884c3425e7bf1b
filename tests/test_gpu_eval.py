"""GPU evaluation (collo_eval) against the oracle on identical seeded inputs."""
import numpy as np
import pytest

from paper_2607_12201_gb300 import workloads as W
from oracle.init import forward_sweep
from oracle.nlp import Problem as OProblem
from gpu_helpers import assemble_J, assemble_W, random_point, rel_max, sparse_rel

pytestmark = pytest.mark.gpu

CASES = {
    "cascade_N50": lambda: W.config1(),
    "tiny_N1": lambda: W.small_network(n=3, r=4, N=1, seed=7),
    "tiny_N5": lambda: W.small_network(n=3, r=5, N=5, seed=8),
    "one_species": lambda: W.random_network(1, 2, n_obs=1, M=5, T=2.0, N=3, seed=9),
    "config2_N400": lambda: W.config2(),
    "config3_N64": lambda: W.config3(N=64),
}


@pytest.fixture(scope="module")
def collo():
    from paper_2607_12201_gb300 import build
    build.build()
    from paper_2607_12201_gb300 import collo
    return collo


@pytest.mark.parametrize("name", list(CASES))
def test_eval_matches_oracle(collo, name):
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


def test_eval_without_multipliers_and_nonfinite_detection(collo):
    inst = W.small_network(n=3, r=4, N=4, seed=3)
    oprob = OProblem(inst)
    x, _ = random_point(oprob, 2)
    with collo.Problem(inst) as prob:
        out = prob.eval(x, None)
        ev = oprob.evaluate(x, np.zeros(oprob.n_c))
        assert rel_max(out["hess_zz"], 0 * out["hess_zz"]) == 0.0
        assert abs(out["phi"] - ev["phi"]) <= 1e-13 * max(1, ev["phi"])
        xb = x.copy()
        xb[5] = np.nan
        with pytest.raises(collo.ColloError) as e:
            prob.eval(xb, None)
        assert e.value.status == collo.ERR_NUMERIC


SWEEP_CASES = {
    # 3n <= 32: the one-warp sweep
    "cascade_N50": CASES["cascade_N50"], "tiny_N5": CASES["tiny_N5"],
    "config2_N400": CASES["config2_N400"],
    # the block sweep: its Jacobian (3n = 39, 90) in shared memory, then
    # (3n = 210) in global memory
    "n13_N20": lambda: W.random_network(13, 26, n_obs=4, M=20, T=5.0, N=20, seed=52,
                                        theta0_spread=0.1),
    "config3_N64": CASES["config3_N64"],
    "n70_N3": lambda: W.random_network(70, 140, n_obs=4, M=12, T=3.0, N=3, seed=71,
                                       theta0_spread=0.1),
}


@pytest.mark.parametrize("name", list(SWEEP_CASES))
def test_forward_sweep_matches_oracle(collo, name):
    inst = SWEEP_CASES[name]()
    oprob = OProblem(inst)
    th = np.array(inst.theta0, dtype=float)
    z_ref, f_ref = forward_sweep(oprob, th)
    with collo.Problem(inst) as prob:
        x, f = prob.initial_states(th)
    assert f == f_ref
    z = x[:oprob.nz].reshape(z_ref.shape)
    assert np.max(np.abs(z - z_ref)) <= 1e-11 * max(1.0, np.max(np.abs(z_ref)))
