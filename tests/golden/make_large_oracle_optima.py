"""Write tests/golden/oracle_optima_large.json: the CPU oracle's optima of the
large parity cases (the stiff 30-species network at its full mesh N = 2000,
instances shaped like the uneven multistart batch and the serving stream, the
members of an uneven batch).

Each of these oracle solves takes minutes to hours on a CPU, far longer than a
GPU test may run, so their results are stored.  This script calls only
``oracle/`` and the seeded input generator; nothing in it comes from the CUDA
path.  The GPU tests (``tests/test_gpu_large.py``) compare the library's
solves of the same seeded instances with these values.

Run from the repository root, one case per process (they are independent):

    OPENBLAS_NUM_THREADS=1 python tests/golden/make_large_oracle_optima.py <case>
    python tests/golden/make_large_oracle_optima.py --list

Single-threaded BLAS is several times faster here: the oracle's block
elimination makes thousands of LAPACK calls on blocks of a few hundred rows.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "oracle_optima_large.json")
TOL = 1e-8
CHECK_BACK = 5


def cases():
    """name -> (instance factory, description).  Starting points lie within
    +-0.1 decade of the true rate constants, where the oracle and the library
    follow the same iterates to the end."""
    from paper_2607_12201_gb300 import workloads as W

    def net(n, N, seed):
        return lambda: W.random_network(n, 2 * n, log10k=(-2.0, 1.0), n_obs=min(4, n), M=50,
                                        T=20.0, N=N, seed=seed, theta0_spread=0.1,
                                        name=f"uneven_n{n}_N{N}_s{seed}")

    out = {
        "config3_N2000": (lambda: W.config3(),
                          "stiff network, 30 species / 60 reactions, 30 estimated, N = 2000"),
        "config4_n50_N100": (net(50, 100, 4001),
                             "multistart-batch shape at its largest species count n = 50 "
                             "(r = p = 100), N = 100"),
        "config5_n100_N40": (net(100, 40, 5001),
                             "serving-stream shape at its largest species count n = 100 "
                             "(r = p = 200), N = 40"),
    }
    for n, N, seed in ((5, 160, 6001), (9, 90, 6002), (14, 120, 6003), (22, 60, 6004),
                       (31, 45, 6005), (40, 30, 6006)):
        out[f"batch_n{n}_N{N}"] = (net(n, N, seed), "member of an uneven batch")
    return out


def solve_case(name):
    from oracle import ipm

    make, desc = cases()[name]
    inst = make()
    t0 = time.time()
    res = ipm.solve(inst, opt=ipm.Options(tol=TOL))
    extra = {}
    if res.status not in (ipm.SUCCESS, ipm.ACCEPTABLE) and res.iterations > 1:
        # a failed solve's last steps are taken near alpha_min, where rounding
        # decides ties in the filter tests: the parity point is the iterate
        # CHECK_BACK iterations before the failure
        m = max(1, res.iterations - CHECK_BACK)
        extra = {"checkpoint_iter": m, "checkpoint_theta": res.history[m - 1]["theta"].tolist(),
                 "trajectory": [h["theta"].tolist() for h in res.history]}
    return {
        "cite": "Eq. 2 NLP solved by the filter line-search interior-point method "
                "(Introduction; tolerances of Section \"Optimization framework configurations\")",
        "description": desc, "instance": inst.name, "n": inst.n, "p": inst.p, "N": inst.N,
        "tol": TOL, "status": int(res.status), "iterations": int(res.iterations),
        "theta": res.x[-inst.p:].tolist(), "phi": float(res.phi),
        "kkt_error": float(res.kkt_error), "cpu_seconds": round(time.time() - t0, 1), **extra}


def merge(name, rec):
    import fcntl
    with open(OUT + ".lock", "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)   # cases run as parallel processes
        data = {}
        if os.path.exists(OUT):
            with open(OUT) as f:
                data = json.load(f)
        data[name] = rec
        with open(OUT, "w") as f:
            json.dump(dict(sorted(data.items())), f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    if len(sys.argv) != 2:
        sys.exit(__doc__)
    if sys.argv[1] == "--list":
        print("\n".join(cases()))
        sys.exit(0)
    rec = solve_case(sys.argv[1])
    merge(sys.argv[1], rec)
    print(sys.argv[1], rec["status"], rec["iterations"], rec["phi"], rec["cpu_seconds"])
