"""Full interior-point solves on the GPU (collo_ipm_solve) against the oracle."""
import numpy as np
import pytest

from paper_2607_12201_gb300 import workloads as W
from oracle import ipm as oipm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def collo():
    from paper_2607_12201_gb300 import build
    build.build()
    from paper_2607_12201_gb300 import collo
    return collo


def _compare(res, ref, inst):
    assert res["status"] == ref.status
    th_ref = ref.x[-inst.p:]
    rel = np.max(np.abs(res["theta"] - th_ref) / np.maximum(np.abs(th_ref), 1e-12))
    assert rel <= 1e-6, (res["theta"], th_ref)
    assert abs(res["phi"] - ref.phi) <= 1e-6 * max(1.0, abs(ref.phi))


def test_cascade_fp64_matches_oracle(collo):
    inst = W.config1()
    ref = oipm.solve(inst)
    with collo.Problem(inst) as prob:
        res = prob.ipm_solve()
    _compare(res, ref, inst)
    assert res["iterations"] == ref.iterations


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_small_network_matches_oracle(collo, prec):
    inst = W.random_network(4, 8, n_obs=3, M=20, T=5.0, N=40, seed=41, theta0_spread=0.1)
    ref = oipm.solve(inst)
    with collo.Problem(inst) as prob:
        res = prob.ipm_solve(precision=collo.MIXED if prec == "mixed" else collo.FP64)
    _compare(res, ref, inst)


def test_config2_fp64_and_mixed_match_oracle(collo):
    inst = W.config2()
    ref = oipm.solve(inst)
    with collo.Problem(inst) as prob:
        r64 = prob.ipm_solve(precision=collo.FP64)
        rmx = prob.ipm_solve(precision=collo.MIXED)
    _compare(r64, ref, inst)
    _compare(rmx, ref, inst)


def test_start_at_optimum_is_trivial(collo):
    inst = W.config1()
    with collo.Problem(inst) as prob:
        first = prob.ipm_solve()
        again = prob.ipm_solve(theta0=first["theta"])
    assert again["status"] == collo.OK
    assert again["iterations"] <= first["iterations"]
