"""The C-ABI library loads and exports every function include/collo.h declares;
host-side argument validation (runs without a GPU: no compute calls)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_12201_gb300 import build
    build.build()
    from paper_2607_12201_gb300 import collo
    return collo


def declared_functions():
    src = open(os.path.join(ROOT, "include", "collo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(collo_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["collo_problem_create", "collo_eval", "collo_kkt_factor", "collo_kkt_solve",
                     "collo_ipm_solve", "collo_problem_destroy", "collo_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    so = C.CDLL(lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_version_and_options_defaults(lib):
    assert "sm_103a" in lib.version()
    o = lib.Problem.ipm_options()
    assert o.tol == 1e-6 and o.acceptable_tol == 1e-4 and o.acceptable_iter == 15


def _structs(lib, inst, K=3, sigma_scale=1.0, t_shift=0.0):
    species = np.unique(inst.obs_s)
    k = dict(react=np.ascontiguousarray(inst.react, np.int32),
             prod=np.ascontiguousarray(inst.prod, np.int32),
             pidx=np.ascontiguousarray(inst.pidx, np.int32), kfix=np.array(inst.kfix, float),
             x0=np.array(inst.x0, float), lo=np.array(inst.theta_lo, float),
             hi=np.array(inst.theta_hi, float), sp=species.astype(np.int32),
             t=np.array(inst.obs_t, float) + t_shift,
             o=np.searchsorted(species, inst.obs_s).astype(np.int32),
             y=np.array(inst.obs_y, float), s=np.array(inst.obs_sigma, float) * sigma_scale)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))
    net = lib.Network(inst.n, inst.r, ip(k["react"]), ip(k["prod"]), ip(k["pidx"]), dp(k["kfix"]),
                      int(inst.logscale), dp(k["x0"]), inst.p, dp(k["lo"]), dp(k["hi"]))
    obs = lib.Observables(len(species), ip(k["sp"]))
    data = lib.Data(inst.M, dp(k["t"]), ip(k["o"]), dp(k["y"]), dp(k["s"]))
    mesh = lib.Mesh(float(inst.T), int(inst.N), K)
    return net, obs, data, mesh, k


@pytest.mark.parametrize("case", ["K4", "sigma0", "t_out"])
def test_create_rejects_bad_arguments_before_touching_the_device(lib, case):
    from paper_2607_12201_gb300 import workloads
    inst = workloads.linear_cascade(N=4)
    kw = {"K4": dict(K=4), "sigma0": dict(sigma_scale=0.0), "t_out": dict(t_shift=100.0)}[case]
    net, obs, data, mesh, keep = _structs(lib, inst, **kw)
    h = C.c_void_p()
    st = lib.lib.collo_problem_create(C.byref(net), C.byref(obs), C.byref(data), C.byref(mesh),
                                      None, C.byref(h))
    assert st == lib.ERR_INVALID_ARG
    assert lib.last_error()
    assert not h.value


def test_calls_on_null_problem_fail_cleanly(lib):
    L = lib.lib
    assert L.collo_eval(None, None, None, 1.0, None) == lib.ERR_INVALID_ARG
    assert L.collo_kkt_factor(None, None, 0.0, 0.0, 0, None) == lib.ERR_INVALID_ARG
    assert L.collo_kkt_solve(None, None, None, 0, 0.0, None) == lib.ERR_INVALID_ARG
    L.collo_problem_destroy(None)


@pytest.mark.parametrize("K,scheme", [(4, 0), (3, 1), (2, 1), (3, 2), (3, -1)])
def test_create_rejects_scheme_and_K_combinations_that_are_not_built(lib, K, scheme):
    """Radau IIA with K = 3 and Gauss-Legendre with K = 4 are built; every
    other (K, scheme) is INVALID_ARG before the device is touched."""
    from paper_2607_12201_gb300 import workloads
    inst = workloads.linear_cascade(N=4)
    net, obs, data, mesh, keep = _structs(lib, inst, K=K)
    mesh.scheme = scheme
    h = C.c_void_p()
    st = lib.lib.collo_problem_create(C.byref(net), C.byref(obs), C.byref(data), C.byref(mesh),
                                      None, C.byref(h))
    assert st == lib.ERR_INVALID_ARG
    assert not h.value


def test_binding_refuses_unknown_scheme_names(lib):
    import dataclasses
    from paper_2607_12201_gb300 import workloads as W
    with pytest.raises(ValueError, match="collocation scheme"):
        lib.Problem(dataclasses.replace(W.linear_cascade(N=4), scheme="lobatto"))


def _unattached_problem(lib, n_x=10, n_c=8, p=2):
    """A binding Problem with a NULL handle: the library refuses every call on
    it before touching a device, so the binding's own checks run on the CPU."""
    pr = object.__new__(lib.Problem)
    pr.h = C.c_void_p()
    pr.n, pr.r, pr.p, pr.N, pr.K = 1, 1, p, 1, 3
    pr.n_x, pr.n_c = n_x, n_c
    pr.inst = None
    return pr


def test_binding_checks_host_array_lengths_before_calling(lib):
    pr = _unattached_problem(lib)
    with pytest.raises(ValueError, match="x has 9 values, expected 10"):
        pr.eval(np.zeros(9))
    with pytest.raises(ValueError, match="lam has 9 values, expected 8"):
        pr.eval(np.zeros(10), np.zeros(9))
    with pytest.raises(ValueError, match="sigma"):
        pr.kkt_factor(np.zeros(11))
    with pytest.raises(ValueError, match="rhs"):
        pr.kkt_solve(np.zeros(17))
    with pytest.raises(ValueError, match="out"):
        pr.kkt_solve(np.zeros(18), out=np.zeros(17))
    with pytest.raises(ValueError, match="theta0"):
        pr.ipm_solve(theta0=np.zeros(3))
    with pytest.raises(ValueError, match="theta"):
        pr.initial_states(np.zeros(1))
    # right lengths reach the library, which refuses the NULL problem
    with pytest.raises(lib.ColloError) as e:
        pr.kkt_solve(np.zeros(18))
    assert e.value.status == lib.ERR_INVALID_ARG


def test_ipm_solve_raises_when_the_call_fails_before_a_result(lib):
    # collo_ipm_solve on a NULL problem returns COLLO_ERR_INVALID_ARG without
    # writing the result; the binding must not report the untouched result
    # (status 0, "solved") as an outcome
    pr = _unattached_problem(lib)
    with pytest.raises(lib.ColloError) as e:
        pr.ipm_solve(theta0=np.zeros(2), want_x=False)
    assert e.value.status == lib.ERR_INVALID_ARG


def test_batch_and_server_check_start_lengths(lib):
    pr = _unattached_problem(lib)
    with pytest.raises(ValueError, match=r"theta0s\[1\]"):
        lib.batch_solve([pr, pr], theta0s=[np.zeros(2), np.zeros(5)])
    sv = object.__new__(lib.Server)
    sv.h, sv._keep = C.c_void_p(), {}
    with pytest.raises(ValueError, match="theta0"):
        sv.submit(pr, theta0=np.zeros(1))
    with pytest.raises(lib.ColloError) as e:       # right length: the NULL server is refused
        sv.submit(pr, theta0=np.zeros(2))
    assert e.value.status == lib.ERR_INVALID_ARG


class _FakeLib:
    """Stands in for the loaded library on the CPU: answers the binding's calls
    the way the C functions do (statuses, outputs written through the result
    pointers) so that the binding's success paths run without a device.  Calls
    it does not define go to the real library (host-only ones such as the
    option defaults)."""

    def __init__(self, real, n_x, n_c, outcome):
        self.real, self.n_x, self.n_c, self.outcome = real, n_x, n_c, outcome
        self.tickets = 0

    def __getattr__(self, name):
        return getattr(self.real, name)

    def collo_eval(self, h, x, lam, of, eo):
        return 0

    def collo_kkt_factor(self, h, sig, dw, dc, prec, inr):
        inr._obj.n_pos, inr._obj.n_neg, inr._obj.n_zero = self.n_x, self.n_c, 0
        return 0

    def collo_kkt_solve(self, h, rhs, sol, rmax, rtol, info):
        C.memmove(sol, rhs, 8 * (self.n_x + self.n_c))
        info._obj.refinement_sweeps = 2
        return 0

    def collo_ipm_solve(self, h, th0, opts, res):
        res._obj.status, res._obj.iterations = self.outcome, 7
        return self.outcome

    def collo_initial_states(self, h, th, x, fails):
        fails._obj.value = 0
        return 0

    def collo_batch_solve(self, handles, n, thp, opts, res):
        for i in range(n):
            res[i].status, res[i].iterations = self.outcome, 5
        return 0

    def collo_server_submit(self, sv, prob, th, ticket):
        self.tickets += 1
        ticket._obj.value = self.tickets
        return 0

    def collo_server_poll(self, sv, ticket, res):
        res._obj.status = self.outcome
        return 0


@pytest.mark.parametrize("outcome", [0, 1, -7, -5])
def test_binding_success_paths(lib, monkeypatch, outcome):
    pr = _unattached_problem(lib)
    monkeypatch.setattr(lib, "lib", _FakeLib(lib.lib, pr.n_x, pr.n_c, outcome))
    pr.eval(np.zeros(10), np.zeros(8), outputs=False)
    ev = pr.eval(np.zeros(10))
    assert ev["phi"] == 0.0 and ev["c"].shape == (8,) and ev["jac_theta"].shape == (1, 3, 1, 2)
    assert pr.kkt_factor(np.zeros(10), 0.0, 1e-8) == (10, 8, 0)
    rhs = np.arange(18.0)
    sol, info = pr.kkt_solve(rhs)
    assert np.array_equal(sol, rhs) and info["sweeps"] == 2
    out = np.empty(18)
    assert pr.kkt_solve(rhs, out=out)[0] is out and np.array_equal(out, rhs)
    r = pr.ipm_solve(theta0=[0.1, 0.2], want_x=True)      # solver outcomes come back as results
    assert r["status"] == outcome and r["iterations"] == 7 and r["x"].shape == (10,)
    x, fails = pr.initial_states([0.1, 0.2])
    assert x.shape == (10,) and fails == 0
    res = lib.batch_solve([pr, pr], theta0s=[[0.0, 0.0], np.ones(2)])
    assert [q["status"] for q in res] == [outcome, outcome]
    sv = object.__new__(lib.Server)
    sv.h, sv._keep = C.c_void_p(), {}
    t = sv.submit(pr, theta0=np.zeros(2))
    assert sv.poll(t)["status"] == outcome


def test_schedule_get_set_and_validation(lib):
    """collo_get_schedule / collo_set_schedule are host-side (no GPU): values
    outside the documented sets are refused and the schedule is unchanged."""
    before = lib.get_schedule()
    assert before["big_threads"] in (256, 512) and before["slab_pairs"] in (8, 16)
    try:
        for bad in (dict(before, big_threads=384), dict(before, slab_pairs=12),
                    dict(before, solve_top_blocks=0), dict(before, solve_elems_per_block=0)):
            with pytest.raises(lib.ColloError) as e:
                lib.set_schedule(bad)
            assert e.value.status == lib.ERR_INVALID_ARG
            assert lib.get_schedule() == before
        other = dict(big_threads=256, slab_pairs=8, solve_top_blocks=16, solve_elems_per_block=4)
        lib.set_schedule(other)
        assert lib.get_schedule() == other
    finally:
        lib.set_schedule(before)


def test_autotune_cache_key_depends_on_shapes_and_device(lib):
    class P:
        def __init__(self, n, p, N):
            self.n, self.p, self.N = n, p, N
    a = [P(5, 10, 100), P(20, 40, 300)]
    b = [P(20, 40, 300), P(5, 10, 100)]
    assert lib.shape_key(a, lib.MIXED, "gpu") == lib.shape_key(b, lib.MIXED, "gpu")
    assert lib.shape_key(a, lib.MIXED, "gpu") != lib.shape_key(a, lib.FP64, "gpu")
    assert lib.shape_key(a, lib.MIXED, "gpu") != lib.shape_key(a, lib.MIXED, "other")
    assert lib.shape_key(a, lib.MIXED, "gpu") != lib.shape_key(a[:1], lib.MIXED, "gpu")
