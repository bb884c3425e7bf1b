"""Write tests/golden/oracle_values.json: reference values of the CPU oracle.

The paper prints no worked example of the method (only its formulas and
whole-solve times), so these values are the oracle's, written by this script,
which calls only ``oracle/`` and the seeded input generator.  They are a
regression anchor: a change to the oracle's arithmetic shows up as a mismatch
in ``tests/test_oracle_golden.py``, and the commit that changes them names the
passage of the paper that justifies it.  The values themselves are pinned by
the independent checks in ``tests/test_oracle_*.py``.

Run from the repository root:  python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


def values():
    from oracle import ipm
    from oracle.radau import Tables
    from paper_2607_12201_gb300 import workloads as W

    out = {}
    for name, K, scheme in (("radau_K3", 3, "radau"), ("gauss_K4", 4, "gauss")):
        t = Tables(K, scheme)
        out[f"tables_{name}"] = {
            "cite": "Eq. 3: interpolation points tau_j and weights d l_j / d tau at tau_k; "
                    "Eq. 2c continuity weights b_j = l_j(1)",
            "tau": t.tau.tolist(), "D": t.D.tolist(), "b": t.b.tolist()}
    solves = {
        "cascade_config1": (W.config1(), ipm.Options(tol=1e-10)),
        "small_network_n3_r4_N6": (W.small_network(n=3, r=4, N=6, seed=7), ipm.Options()),
    }
    for name, (inst, opt) in solves.items():
        r = ipm.solve(inst, opt=opt)
        out[f"ipm_{name}"] = {
            "cite": "Eq. 2 NLP solved by the filter line-search interior-point method "
                    "(Introduction; tolerances of Section \"Optimization framework configurations\")",
            "tol": opt.tol, "status": int(r.status), "iterations": int(r.iterations),
            "theta": r.x[-inst.p:].tolist(), "phi": float(r.phi)}
    return out


if __name__ == "__main__":
    path = os.path.join(HERE, "oracle_values.json")
    with open(path, "w") as f:
        json.dump(values(), f, indent=1)
        f.write("\n")
    print("wrote", path)
