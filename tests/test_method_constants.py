"""The CUDA interior-point driver and the oracle state the constants of
Waechter & Biegler (2006) independently (they share no code); this CPU test
reads the driver's defaults from its source and holds them equal to the
oracle's, and the library's default options to the oracle's tolerances."""
import os
import re

import pytest

from oracle import ipm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# CUDA driver name -> oracle Options field
NAMES = {
    "mu_init": "mu_init", "kappa_mu": "kappa_mu", "theta_mu": "theta_mu",
    "kappa_eps": "kappa_eps", "tau_min": "tau_min", "s_max": "s_max",
    "kappa1": "bound_push", "kappa2": "bound_frac", "kappa_sigma": "kappa_sigma",
    "gamma_theta": "gamma_theta", "gamma_phi": "gamma_phi", "delta": "delta",
    "s_theta": "s_theta", "s_phi": "s_phi", "eta_phi": "eta_phi",
    "gamma_alpha": "gamma_alpha", "dw_min": "dw_min", "dw_0": "dw_0", "dw_max": "dw_max",
    "kw_minus": "kw_minus", "kw_plus": "kw_plus", "kw_plus_bar": "kw_plus_bar",
    "dc_coef": "dc_coef", "dc_exp": "dc_exp",
}


def driver_constants():
    src = open(os.path.join(ROOT, "paper_2607_12201_gb300", "csrc", "runner.cu")).read()
    body = re.search(r"struct Opt \{(.*?)\};", src, flags=re.S).group(1)
    found = {}
    for name, expr in re.findall(r"(\w+) = ([0-9eE.+\-/ ]+?)[,;]", body):
        found[name] = eval(expr, {"__builtins__": {}})      # numeric literals and one division
    return found


def test_driver_states_every_constant_once():
    found = driver_constants()
    assert set(found) == set(NAMES)


@pytest.mark.parametrize("cuda_name", sorted(NAMES))
def test_driver_constant_equals_the_oracle_s(cuda_name):
    assert driver_constants()[cuda_name] == getattr(ipm.Options(), NAMES[cuda_name])


def test_library_default_tolerances_equal_the_oracle_s():
    from paper_2607_12201_gb300 import build
    build.build()
    from paper_2607_12201_gb300 import collo
    o, ref = collo.Problem.ipm_options(), ipm.Options()
    assert (o.tol, o.acceptable_tol, o.acceptable_iter) == (ref.tol, ref.acceptable_tol,
                                                            ref.acceptable_iter)
