"""Thin ctypes binding of libcollo (include/collo.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy
arrays / raw device pointers to the C structures and back.  Importing it
loads ``libcollo.so`` and fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcollo.so")

OK, ACCEPTABLE = 0, 1
ERR_INVALID_ARG, ERR_OOM, ERR_NUMERIC, ERR_INERTIA = -1, -2, -3, -4
ERR_MAXITER, ERR_TIMEOUT, ERR_LINESEARCH, ERR_NOT_FACTORED = -5, -6, -7, -8
ERR_DEVICE, ERR_NOT_EVALUATED = -9, -10
PENDING = 2
FP64, MIXED = 0, 1


class ColloError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"collo status {status}: {msg}")
        self.status = status


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class Network(C.Structure):
    _fields_ = [("n_species", C.c_int), ("n_reactions", C.c_int), ("reactants", _ip),
                ("products", _ip), ("param_index", _ip), ("k_fixed", _dp),
                ("log10_params", C.c_int), ("x0", _dp), ("n_params", C.c_int),
                ("theta_lo", _dp), ("theta_hi", _dp)]


class Observables(C.Structure):
    _fields_ = [("n_observables", C.c_int), ("species", _ip)]


class Data(C.Structure):
    _fields_ = [("n_obs", C.c_int), ("t", _dp), ("observable", _ip), ("y", _dp), ("sigma", _dp)]


SCHEME_RADAU, SCHEME_GAUSS = 0, 1
_SCHEMES = {"radau": SCHEME_RADAU, "gauss": SCHEME_GAUSS}


class Mesh(C.Structure):
    _fields_ = [("T", C.c_double), ("N", C.c_int), ("K", C.c_int), ("scheme", C.c_int)]


class Conditions(C.Structure):
    _fields_ = [("n_conditions", C.c_int), ("x0", _dp), ("rate_scale", _dp),
                ("obs_condition", _ip)]


class ProblemOptions(C.Structure):
    _fields_ = [("precision", C.c_int), ("stream", C.c_void_p), ("device", C.c_int),
                ("launch_mode", C.c_int), ("reserved", C.c_int * 6)]


class Sizes(C.Structure):
    _fields_ = [("n", C.c_int), ("r", C.c_int), ("p", C.c_int), ("N", C.c_int), ("K", C.c_int),
                ("M", C.c_int), ("n_x", C.c_int64), ("n_c", C.c_int64), ("levels", C.c_int),
                ("device_bytes", C.c_int64), ("n_conditions", C.c_int),
                ("elements_per_condition", C.c_int)]


class EvalOut(C.Structure):
    _fields_ = [(name, C.c_void_p) for name in
                ["phi", "c", "grad", "jac_z", "jac_theta", "hess_zz", "hess_ztheta", "hess_thth",
                 "hess_obj"]]


class Inertia(C.Structure):
    _fields_ = [("n_pos", C.c_int64), ("n_neg", C.c_int64), ("n_zero", C.c_int64)]


class SolveInfo(C.Structure):
    _fields_ = [("refinement_sweeps", C.c_int), ("residual", C.c_double)]


class IpmOptions(C.Structure):
    _fields_ = [("tol", C.c_double), ("acceptable_tol", C.c_double), ("acceptable_iter", C.c_int),
                ("max_iter", C.c_int), ("max_wall_time", C.c_double), ("precision", C.c_int),
                ("mixed_mu_switch", C.c_double), ("refine_max", C.c_int),
                ("refine_tol", C.c_double), ("verbose", C.c_int), ("reserved", C.c_int * 8)]


class Schedule(C.Structure):
    _fields_ = [("big_threads", C.c_int), ("slab_pairs", C.c_int), ("solve_top_blocks", C.c_int),
                ("solve_elems_per_block", C.c_int), ("reserved", C.c_int * 4)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("factorizations", C.c_int),
                ("line_search_trials", C.c_int), ("refinement_sweeps", C.c_int),
                ("fp64_factorizations", C.c_int), ("phi", C.c_double), ("kkt_error", C.c_double),
                ("mu", C.c_double), ("wall_seconds", C.c_double), ("theta", C.c_void_p),
                ("x", C.c_void_p), ("lambda_", C.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_2607_12201_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    lib.collo_problem_create.argtypes = [C.POINTER(Network), C.POINTER(Observables),
                                         C.POINTER(Data), C.POINTER(Mesh),
                                         C.POINTER(ProblemOptions), C.POINTER(P)]
    lib.collo_problem_create.restype = C.c_int
    lib.collo_problem_create_conditions.argtypes = [
        C.POINTER(Network), C.POINTER(Observables), C.POINTER(Data), C.POINTER(Mesh),
        C.POINTER(Conditions), C.POINTER(ProblemOptions), C.POINTER(P)]
    lib.collo_problem_create_conditions.restype = C.c_int
    lib.collo_problem_destroy.argtypes = [P]
    lib.collo_problem_destroy.restype = None
    lib.collo_problem_sizes.argtypes = [P, C.POINTER(Sizes)]
    lib.collo_problem_sizes.restype = C.c_int
    lib.collo_problem_stream.argtypes = [P]
    lib.collo_problem_stream.restype = C.c_void_p
    lib.collo_problem_solve_bytes.argtypes = [P, C.c_int, C.POINTER(C.c_int64)]
    lib.collo_problem_solve_bytes.restype = C.c_int
    lib.collo_problem_set_wait_limit.argtypes = [P, C.c_longlong, C.c_int]
    lib.collo_problem_set_wait_limit.restype = C.c_int
    lib.collo_eval.argtypes = [P, C.c_void_p, C.c_void_p, C.c_double, C.POINTER(EvalOut)]
    lib.collo_eval.restype = C.c_int
    lib.collo_kkt_factor.argtypes = [P, C.c_void_p, C.c_double, C.c_double, C.c_int,
                                     C.POINTER(Inertia)]
    lib.collo_kkt_factor.restype = C.c_int
    lib.collo_kkt_solve.argtypes = [P, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                    C.POINTER(SolveInfo)]
    lib.collo_kkt_solve.restype = C.c_int
    lib.collo_lifted_factor.argtypes = [P, C.c_void_p, C.c_void_p, C.c_double,
                                        C.POINTER(C.c_int)]
    lib.collo_lifted_factor.restype = C.c_int
    lib.collo_lifted_solve.argtypes = [P, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                       C.POINTER(SolveInfo)]
    lib.collo_lifted_solve.restype = C.c_int
    lib.collo_lifted_ipm_solve.argtypes = [P, C.c_void_p, C.c_double, C.POINTER(IpmOptions),
                                           C.POINTER(Result)]
    lib.collo_lifted_ipm_solve.restype = C.c_int
    lib.collo_ipm_options_default.argtypes = [C.POINTER(IpmOptions)]
    lib.collo_ipm_options_default.restype = None
    lib.collo_ipm_solve.argtypes = [P, C.c_void_p, C.POINTER(IpmOptions), C.POINTER(Result)]
    lib.collo_ipm_solve.restype = C.c_int
    lib.collo_initial_states.argtypes = [P, C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]
    lib.collo_initial_states.restype = C.c_int
    lib.collo_eval_noalloc.argtypes = [P, C.c_void_p, C.c_void_p, C.c_double,
                                        C.POINTER(EvalOut), C.c_void_p]
    lib.collo_eval_noalloc.restype = C.c_int
    lib.collo_batch_solve.argtypes = [C.POINTER(P), C.c_int, C.POINTER(C.c_void_p),
                                       C.POINTER(IpmOptions), C.POINTER(Result)]
    lib.collo_batch_solve.restype = C.c_int
    lib.collo_batch_time_phase.argtypes = [C.POINTER(P), C.c_int, C.c_int, C.c_int, C.c_int,
                                           C.POINTER(C.c_double)]
    lib.collo_batch_time_phase.restype = C.c_int
    lib.collo_server_create.argtypes = [C.c_int, C.c_int64, C.POINTER(IpmOptions), C.c_int,
                                        C.POINTER(P)]
    lib.collo_server_create.restype = C.c_int
    lib.collo_server_submit.argtypes = [P, P, C.c_void_p, C.POINTER(C.c_longlong)]
    lib.collo_server_submit.restype = C.c_int
    lib.collo_server_step.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.collo_server_step.restype = C.c_int
    lib.collo_server_poll.argtypes = [P, C.c_longlong, C.POINTER(Result)]
    lib.collo_server_poll.restype = C.c_int
    lib.collo_server_destroy.argtypes = [P]
    lib.collo_server_destroy.restype = None
    lib.collo_server_set_admission.argtypes = [P, C.c_int]
    lib.collo_server_set_admission.restype = C.c_int
    lib.collo_phase_profile.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.c_int,
                                        C.c_int]
    lib.collo_phase_profile.restype = C.c_int
    lib.collo_server_stream.argtypes = [P]
    lib.collo_server_stream.restype = C.c_void_p
    lib.collo_server_memory.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.collo_server_memory.restype = C.c_int
    lib.collo_server_counters.argtypes = [P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                          C.POINTER(C.c_longlong)]
    lib.collo_server_counters.restype = C.c_int
    lib.collo_time_phase.argtypes = [P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]
    lib.collo_time_phase.restype = C.c_int
    lib.collo_problem_create_refined.argtypes = [P, C.c_int, C.POINTER(P)]
    lib.collo_problem_create_refined.restype = C.c_int
    lib.collo_defect.argtypes = [P, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]
    lib.collo_defect.restype = C.c_int
    lib.collo_interpolate.argtypes = [P, C.c_void_p, P, C.c_void_p]
    lib.collo_interpolate.restype = C.c_int
    lib.collo_problem_set_start.argtypes = [P, C.c_void_p, C.c_void_p]
    lib.collo_problem_set_start.restype = C.c_int
    lib.collo_refine_solve.argtypes = [C.POINTER(P), C.c_int, C.POINTER(C.c_void_p),
                                       C.POINTER(IpmOptions), C.c_double, C.c_int, C.c_int,
                                       C.POINTER(P), C.POINTER(Result), C.POINTER(C.c_int)]
    lib.collo_refine_solve.restype = C.c_int
    lib.collo_get_schedule.argtypes = [C.POINTER(Schedule)]
    lib.collo_get_schedule.restype = C.c_int
    lib.collo_set_schedule.argtypes = [C.POINTER(Schedule)]
    lib.collo_set_schedule.restype = C.c_int
    lib.collo_autotune.argtypes = [C.POINTER(P), C.c_int, C.c_int, C.c_int, C.POINTER(Schedule),
                                   C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.collo_autotune.restype = C.c_int
    lib.collo_alu_peak.argtypes = [C.c_int, C.POINTER(C.c_double)]
    lib.collo_alu_peak.restype = C.c_int
    lib.collo_launch_count.argtypes = []
    lib.collo_launch_count.restype = C.c_longlong
    lib.collo_last_error.argtypes = []
    lib.collo_last_error.restype = C.c_char_p
    lib.collo_version.argtypes = []
    lib.collo_version.restype = C.c_char_p
    return lib


lib = _load()


def last_error() -> str:
    return lib.collo_last_error().decode()


def _check(status, allow=(OK,)):
    if status not in allow:
        raise ColloError(status, last_error())
    return status


def _ptr(a):
    """Address of a numpy array, a torch tensor or an int (device pointer)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays passed to the library must be C-contiguous")
        return a.ctypes.data
    return int(a.data_ptr())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _host_vec(a, size, what):
    """A host array of exactly ``size`` doubles (converted, length checked: the
    library reads ``size`` values through the pointer).  ``None``, an int
    (a raw pointer) or a tensor pass through unchecked: their extent is the
    caller's responsibility."""
    if a is None or isinstance(a, int) or hasattr(a, "data_ptr"):
        return a
    v = np.ascontiguousarray(a, dtype=np.float64)
    if v.size != size:
        raise ValueError(f"{what} has {v.size} values, expected {size}")
    return v


# statuses of a call that failed as a call (not an outcome of the solve)
_CALL_ERRORS = (ERR_INVALID_ARG, ERR_OOM, ERR_NOT_FACTORED, ERR_DEVICE, ERR_NOT_EVALUATED)


class Problem:
    """One estimation problem resident on the GPU (wraps collo_problem)."""

    def __init__(self, inst, precision: int = FP64, stream: int | None = None, device: int = 0,
                 launch_mode: int = 0):
        self.inst = inst
        scheme = getattr(inst, "scheme", "radau")
        if scheme not in _SCHEMES:
            raise ValueError(f"unknown collocation scheme {scheme!r}")
        species = np.unique(inst.obs_s)
        obs_index = np.searchsorted(species, inst.obs_s)
        self._keep = dict(
            react=_i32(inst.react), prod=_i32(inst.prod), pidx=_i32(inst.pidx),
            kfix=_f64(inst.kfix), x0=_f64(inst.x0), lo=_f64(inst.theta_lo),
            hi=_f64(inst.theta_hi), species=_i32(species), t=_f64(inst.obs_t),
            obs=_i32(obs_index), y=_f64(inst.obs_y), sig=_f64(inst.obs_sigma))
        k = self._keep
        dp = lambda a: a.ctypes.data_as(_dp)
        ip = lambda a: a.ctypes.data_as(_ip)
        net = Network(inst.n, inst.r, ip(k["react"]), ip(k["prod"]), ip(k["pidx"]), dp(k["kfix"]),
                      int(inst.logscale), dp(k["x0"]), inst.p, dp(k["lo"]), dp(k["hi"]))
        obs = Observables(len(species), ip(k["species"]))
        data = Data(inst.M, dp(k["t"]), ip(k["obs"]), dp(k["y"]), dp(k["sig"]))
        mesh = Mesh(float(inst.T), int(inst.N), int(inst.K), _SCHEMES[scheme])
        opt = ProblemOptions(precision, stream, device, launch_mode)
        h = C.c_void_p()
        if getattr(inst, "cond_x0", None) is not None:
            k["cx0"] = _f64(inst.cond_x0).reshape(-1)
            k["csc"] = (_f64(inst.cond_scale).reshape(-1)
                        if getattr(inst, "cond_scale", None) is not None else None)
            k["oc"] = (_i32(inst.obs_cond) if getattr(inst, "obs_cond", None) is not None
                       else None)
            cond = Conditions(inst.Nc, dp(k["cx0"]),
                              dp(k["csc"]) if k["csc"] is not None else None,
                              ip(k["oc"]) if k["oc"] is not None else None)
            _check(lib.collo_problem_create_conditions(
                C.byref(net), C.byref(obs), C.byref(data), C.byref(mesh), C.byref(cond),
                C.byref(opt), C.byref(h)))
        else:
            _check(lib.collo_problem_create(C.byref(net), C.byref(obs), C.byref(data),
                                            C.byref(mesh), C.byref(opt), C.byref(h)))
        self.h = h
        s = Sizes()
        _check(lib.collo_problem_sizes(self.h, C.byref(s)))
        self.sizes = s
        self.n, self.r, self.p, self.N, self.K = s.n, s.r, s.p, s.N, s.K
        self.Nc, self.Nch = s.n_conditions, s.elements_per_condition
        self.n_x, self.n_c = int(s.n_x), int(s.n_c)

    @classmethod
    def _adopt(cls, handle, inst):
        """Wrap a problem the library created (the wrapper owns it)."""
        self = cls.__new__(cls)
        self.inst = inst
        self._keep = {}
        self.h = C.c_void_p(handle) if not isinstance(handle, C.c_void_p) else handle
        s = Sizes()
        _check(lib.collo_problem_sizes(self.h, C.byref(s)))
        self.sizes = s
        self.n, self.r, self.p, self.N, self.K = s.n, s.r, s.p, s.N, s.K
        self.Nc, self.Nch = s.n_conditions, s.elements_per_condition
        self.n_x, self.n_c = int(s.n_x), int(s.n_c)
        return self

    def refined(self, N: int) -> "Problem":
        """collo_problem_create_refined: the same problem on N elements."""
        h = C.c_void_p()
        _check(lib.collo_problem_create_refined(self.h, int(N), C.byref(h)))
        return Problem._adopt(h, self.inst.with_mesh(N))

    def defect(self, x):
        """collo_defect: (per-element defects [N], their maximum)."""
        x = _host_vec(x, self.n_x, "x")
        d = np.zeros(self.N)
        mx = C.c_double()
        _check(lib.collo_defect(self.h, _ptr(x), d.ctypes.data, C.byref(mx)))
        return d, mx.value

    def set_start(self, x, lam=None):
        """collo_problem_set_start: warm start of the next solve (x = None clears)."""
        x = _host_vec(x, self.n_x, "x") if x is not None else None
        lam = _host_vec(lam, self.n_c, "lam") if lam is not None else None
        _check(lib.collo_problem_set_start(self.h, _ptr(x), _ptr(lam)))

    def close(self):
        if getattr(self, "h", None):
            lib.collo_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def stream(self) -> int:
        return lib.collo_problem_stream(self.h)

    def device_bytes(self) -> int:
        """Device bytes the problem holds now (collo_problem_sizes)."""
        s = Sizes()
        _check(lib.collo_problem_sizes(self.h, C.byref(s)))
        return int(s.device_bytes)

    def solve_bytes(self, precision: int = FP64) -> int:
        """collo_problem_solve_bytes: device bytes held while a solve runs."""
        b = C.c_int64()
        _check(lib.collo_problem_solve_bytes(self.h, int(precision), C.byref(b)))
        return int(b.value)

    def set_wait_limit(self, max_polls: int = 0, unreachable: bool = False):
        """collo_problem_set_wait_limit: bound of the grid-barrier waits (0: default)
        and the failure-test switch that makes every barrier unreachable."""
        _check(lib.collo_problem_set_wait_limit(self.h, int(max_polls), int(bool(unreachable))))

    # --- evaluation ------------------------------------------------------------
    def eval(self, x, lam=None, obj_factor: float = 1.0, outputs: bool = True):
        """collo_eval on host arrays; returns a dict of host arrays."""
        n, p, N, K = self.n, self.p, self.N, self.K
        x = _host_vec(x, self.n_x, "x")
        lam = _host_vec(lam, self.n_c, "lam")
        out = {}
        eo = EvalOut()
        if outputs:
            shapes = dict(phi=(1,), c=(self.n_c,), grad=(self.n_x,), jac_z=(N, K, n, n),
                          jac_theta=(N, K, n, p), hess_zz=(N, K, n, n),
                          hess_ztheta=(N, K, n, p), hess_thth=(p,),
                          hess_obj=(N, n, K + 1, K + 1))
            for name, shp in shapes.items():
                out[name] = np.zeros(shp)
                setattr(eo, name, out[name].ctypes.data)
        st = lib.collo_eval(self.h, _ptr(x), _ptr(lam), float(obj_factor), C.byref(eo))
        _check(st)
        if outputs:
            out["phi"] = float(out["phi"][0])
        return out

    def eval_noalloc(self, x_ptr: int, lam_ptr, out_ptrs: dict, obj_factor: float = 1.0,
                     stream: int | None = None):
        """collo_eval_noalloc on device pointers (ints); out_ptrs maps the
        collo_eval_out field names to device pointers.  Asynchronous."""
        eo = EvalOut()
        for name, ptr in out_ptrs.items():
            setattr(eo, name, ptr)
        return _check(lib.collo_eval_noalloc(self.h, x_ptr, lam_ptr, float(obj_factor),
                                             C.byref(eo), stream))

    def eval_raw(self, x_ptr, lam_ptr, obj_factor=1.0):
        """collo_eval on raw (device or host) pointers, no outputs copied."""
        return _check(lib.collo_eval(self.h, x_ptr, lam_ptr, float(obj_factor), None))

    # --- KKT ---------------------------------------------------------------------
    def kkt_factor(self, sigma=None, delta_w=0.0, delta_c=0.0, precision: int = -1):
        inr = Inertia()
        sig = _host_vec(sigma, self.n_x, "sigma")
        _check(lib.collo_kkt_factor(self.h, _ptr(sig), float(delta_w), float(delta_c),
                                    int(precision), C.byref(inr)))
        return (int(inr.n_pos), int(inr.n_neg), int(inr.n_zero))

    def kkt_solve(self, rhs, refine_max: int = 10, refine_tol: float = 1e-12, out=None):
        info = SolveInfo()
        rhs = _host_vec(rhs, self.n_x + self.n_c, "rhs")
        if isinstance(rhs, np.ndarray):
            sol = np.zeros_like(rhs) if out is None else out
        else:
            sol = out
        if isinstance(sol, np.ndarray) and (sol.size != self.n_x + self.n_c
                                            or sol.dtype != np.float64
                                            or not sol.flags.c_contiguous):
            raise ValueError("out must be a contiguous float64 array of the rhs's size")
        _check(lib.collo_kkt_solve(self.h, _ptr(rhs), _ptr(sol), int(refine_max),
                                   float(refine_tol), C.byref(info)))
        return sol, dict(sweeps=info.refinement_sweeps, residual=info.residual)

    def lifted_factor(self, sigma_x, sigma_s, delta_w=0.0) -> bool:
        """Cholesky of the lifted condensed matrix of the last eval; True when
        it is positive definite."""
        sx = _host_vec(sigma_x, self.n_x, "sigma_x")
        ss = _host_vec(sigma_s, self.n_c, "sigma_s")
        if ss is None:
            raise ValueError("sigma_s is required")
        pd = C.c_int(0)
        _check(lib.collo_lifted_factor(self.h, _ptr(sx), _ptr(ss), float(delta_w), C.byref(pd)))
        return bool(pd.value)

    def lifted_solve(self, r_x, r_s, r_c, refine_max: int = 10, refine_tol: float = 1e-12):
        """(dx, ds, dlam) of the lifted system with the last lifted_factor."""
        rx = _host_vec(r_x, self.n_x, "r_x")
        rs = _host_vec(r_s, self.n_c, "r_s")
        rc = _host_vec(r_c, self.n_c, "r_c")
        if rx is None or rs is None or rc is None:
            raise ValueError("r_x, r_s and r_c are required")
        dx, ds, dl = np.zeros(self.n_x), np.zeros(self.n_c), np.zeros(self.n_c)
        info = SolveInfo()
        _check(lib.collo_lifted_solve(self.h, _ptr(rx), _ptr(rs), _ptr(rc), _ptr(dx), _ptr(ds),
                                      _ptr(dl), int(refine_max), float(refine_tol),
                                      C.byref(info)))
        return dx, ds, dl, dict(sweeps=info.refinement_sweeps, residual=info.residual)

    # --- solver ------------------------------------------------------------------
    @staticmethod
    def ipm_options(**kw) -> IpmOptions:
        o = IpmOptions()
        lib.collo_ipm_options_default(C.byref(o))
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    def ipm_solve(self, theta0=None, want_x: bool = True, **kw):
        th0 = _host_vec(_f64(self.inst.theta0 if theta0 is None else theta0), self.p, "theta0")
        o = self.ipm_options(**kw)
        res = Result()
        theta = np.zeros(self.p)
        x = np.zeros(self.n_x) if want_x else None
        lam = np.zeros(self.n_c) if want_x else None
        res.theta = theta.ctypes.data
        res.x = None if x is None else x.ctypes.data
        res.lambda_ = None if lam is None else lam.ctypes.data
        st = lib.collo_ipm_solve(self.h, th0.ctypes.data, C.byref(o), C.byref(res))
        # the call returns the solve's outcome, which it also stores in the result;
        # a call that failed before producing a result returns its error only
        if st in _CALL_ERRORS or st != res.status:
            raise ColloError(st, last_error())
        return _result_dict(res, theta, x, lam)

    def lifted_ipm_solve(self, theta0=None, relax: float = 1e-8, want_x: bool = True, **kw):
        """collo_lifted_ipm_solve: the relaxed-equality form's interior-point solve."""
        th0 = _host_vec(_f64(self.inst.theta0 if theta0 is None else theta0), self.p, "theta0")
        o = self.ipm_options(**kw)
        res = Result()
        theta = np.zeros(self.p)
        x = np.zeros(self.n_x) if want_x else None
        lam = np.zeros(self.n_c) if want_x else None
        res.theta = theta.ctypes.data
        res.x = None if x is None else x.ctypes.data
        res.lambda_ = None if lam is None else lam.ctypes.data
        st = lib.collo_lifted_ipm_solve(self.h, th0.ctypes.data, float(relax), C.byref(o),
                                        C.byref(res))
        if st in _CALL_ERRORS or st != res.status:
            raise ColloError(st, last_error())
        return _result_dict(res, theta, x, lam)

    def time_phase(self, phase: int, precision: int = -1, reps: int = 20) -> float:
        """Average milliseconds per launch of one phase (see collo_time_phase)."""
        ms = C.c_double()
        _check(lib.collo_time_phase(self.h, int(phase), int(precision), int(reps), C.byref(ms)))
        return ms.value

    def initial_states(self, theta):
        x = np.zeros(self.n_x)
        f = C.c_int(0)
        theta = _host_vec(_f64(theta), self.p, "theta")
        _check(lib.collo_initial_states(self.h, theta.ctypes.data, x.ctypes.data,
                                        C.byref(f)))
        return x, int(f.value)


def _result_dict(res, theta, x, lam):
    return dict(status=res.status, iterations=res.iterations, factorizations=res.factorizations,
                trials=res.line_search_trials, refine=res.refinement_sweeps,
                fp64_facs=res.fp64_factorizations, phi=res.phi,
                kkt_error=res.kkt_error, mu=res.mu, wall=res.wall_seconds, theta=theta, x=x,
                lam=lam)


def batch_solve(problems, theta0s=None, want_x: bool = False, **kw):
    """collo_batch_solve: solve several problems together; list of result dicts."""
    n = len(problems)
    handles = (C.c_void_p * n)(*[p.h.value for p in problems])
    th = [_host_vec(_f64(p.inst.theta0 if theta0s is None else theta0s[i]), p.p, f"theta0s[{i}]")
          for i, p in enumerate(problems)]
    thp = (C.c_void_p * n)(*[t.ctypes.data for t in th])
    res = (Result * n)()
    outs = []
    for i, p in enumerate(problems):
        theta = np.zeros(p.p)
        x = np.zeros(p.n_x) if want_x else None
        lam = np.zeros(p.n_c) if want_x else None
        res[i].theta = theta.ctypes.data
        res[i].x = None if x is None else x.ctypes.data
        res[i].lambda_ = None if lam is None else lam.ctypes.data
        outs.append((theta, x, lam))
    o = Problem.ipm_options(**kw)
    _check(lib.collo_batch_solve(handles, n, thp, C.byref(o), res))
    return [_result_dict(res[i], *outs[i]) for i in range(n)]


def interpolate(coarse, x_coarse, fine):
    """collo_interpolate: the coarse solution on fine's mesh (host array)."""
    xc = _host_vec(x_coarse, coarse.n_x, "x_coarse")
    xf = np.zeros(fine.n_x)
    _check(lib.collo_interpolate(coarse.h, _ptr(xc), fine.h, xf.ctypes.data))
    return xf


def refine_solve(problems, theta0s=None, defect_tol: float = 1e-6, max_levels: int = 3,
                 max_elements: int = 0, **kw):
    """collo_refine_solve: batched solve, then refine the converged problems whose
    defect exceeds defect_tol (twice the elements, warm start) up to max_levels
    times.  Returns (results, final problems, levels); a final problem the
    library created is wrapped (and owned) here."""
    n = len(problems)
    handles = (C.c_void_p * n)(*[p.h.value for p in problems])
    th = [_host_vec(_f64(p.inst.theta0 if theta0s is None else theta0s[i]), p.p, f"theta0s[{i}]")
          for i, p in enumerate(problems)]
    thp = (C.c_void_p * n)(*[t.ctypes.data for t in th])
    res = (Result * n)()
    thetas = []
    for i, p in enumerate(problems):
        theta = np.zeros(p.p)
        res[i].theta = theta.ctypes.data
        thetas.append(theta)
    finals = (C.c_void_p * n)()
    levels = (C.c_int * n)()
    o = Problem.ipm_options(**kw)
    _check(lib.collo_refine_solve(handles, n, thp, C.byref(o), float(defect_tol), int(max_levels),
                                  int(max_elements), finals, res, levels))
    out_probs = []
    for i, p in enumerate(problems):
        if finals[i] == p.h.value:
            out_probs.append(p)
        else:
            size = Sizes()
            _check(lib.collo_problem_sizes(C.c_void_p(finals[i]), C.byref(size)))
            out_probs.append(Problem._adopt(finals[i],
                                            p.inst.with_mesh(size.elements_per_condition)))
    return ([_result_dict(res[i], thetas[i], None, None) for i in range(n)], out_probs,
            [int(levels[i]) for i in range(n)])


def batch_time_phase(problems, phase: int, precision: int, reps: int = 10) -> float:
    """collo_batch_time_phase: ms per batched launch of phase 1..7 (factor, solve,
    eval, element condensation alone, reduction + Schur alone, large element
    blocks alone, register-tiled element blocks alone)."""
    n = len(problems)
    handles = (C.c_void_p * n)(*[p.h.value for p in problems])
    ms = C.c_double()
    _check(lib.collo_batch_time_phase(handles, n, int(phase), int(precision), int(reps),
                                      C.byref(ms)))
    return ms.value


SCHEDULE_FIELDS = ["big_threads", "slab_pairs", "solve_top_blocks", "solve_elems_per_block"]


def get_schedule() -> dict:
    """collo_get_schedule: the process-wide launch schedule."""
    sc = Schedule()
    _check(lib.collo_get_schedule(C.byref(sc)))
    return {k: int(getattr(sc, k)) for k in SCHEDULE_FIELDS}


def set_schedule(sched: dict):
    """collo_set_schedule from a dict with the fields of collo_schedule."""
    sc = Schedule()
    for k in SCHEDULE_FIELDS:
        setattr(sc, k, int(sched[k]))
    _check(lib.collo_set_schedule(C.byref(sc)))


def shape_key(problems, precision: int, device_name: str = "") -> str:
    """Cache key of a batch for the autotuner: the device, the precision and
    the sorted (n, p, N) shapes of its problems."""
    import hashlib
    shapes = sorted((p.n, p.p, p.N) for p in problems)
    h = hashlib.sha1(repr((device_name, int(precision), shapes)).encode()).hexdigest()[:16]
    return f"{device_name}|{int(precision)}|{len(shapes)}|{h}"


def autotune(problems, precision: int = MIXED, reps: int = 2, cache: str | None = None,
             device_name: str = ""):
    """collo_autotune over evaluated problems; with `cache` (a JSON file path)
    a batch already tuned on this device reuses the stored schedule.  Returns
    (schedule dict, ms before, ms after, from_cache)."""
    import json
    key = shape_key(problems, precision, device_name)
    table = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
        if key in table:
            ent = table[key]
            set_schedule(ent["schedule"])
            return ent["schedule"], ent["ms_before"], ent["ms_after"], True
    n = len(problems)
    handles = (C.c_void_p * n)(*[p.h.value for p in problems])
    sc = Schedule()
    b, a = C.c_double(), C.c_double()
    _check(lib.collo_autotune(handles, n, int(precision), int(reps), C.byref(sc), C.byref(b),
                              C.byref(a)))
    best = {k: int(getattr(sc, k)) for k in SCHEDULE_FIELDS}
    if cache:
        table[key] = {"schedule": best, "ms_before": b.value, "ms_after": a.value}
        os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
        with open(cache, "w") as f:
            json.dump(table, f, indent=1)
    return best, b.value, a.value, False


class Server:
    """collo_server_*: continuous batching of IPM solves on one GPU."""

    def __init__(self, max_slots: int, budget_bytes: int = 0, device: int = 0, **kw):
        o = Problem.ipm_options(**kw)
        h = C.c_void_p()
        _check(lib.collo_server_create(int(max_slots), int(budget_bytes), C.byref(o), int(device),
                                       C.byref(h)))
        self.h = h
        self._keep = {}

    def submit(self, problem, theta0=None) -> int:
        th = _host_vec(_f64(problem.inst.theta0 if theta0 is None else theta0), problem.p,
                       "theta0")
        t = C.c_longlong()
        _check(lib.collo_server_submit(self.h, problem.h, th.ctypes.data, C.byref(t)))
        self._keep[t.value] = (problem, th)
        return t.value

    def step(self):
        a, w = C.c_int(), C.c_int()
        _check(lib.collo_server_step(self.h, C.byref(a), C.byref(w)))
        return a.value, w.value

    def set_admission(self, min_free_slots: int):
        _check(lib.collo_server_set_admission(self.h, int(min_free_slots)))

    @property
    def stream(self) -> int:
        return int(lib.collo_server_stream(self.h) or 0)

    def counters(self):
        """(Newton steps taken, jobs finished, jobs solved) since creation."""
        a, b, c = C.c_longlong(), C.c_longlong(), C.c_longlong()
        _check(lib.collo_server_counters(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return int(a.value), int(b.value), int(c.value)

    def memory(self):
        """(bytes held by admitted problems now, most held at once so far)."""
        a, pk = C.c_int64(), C.c_int64()
        _check(lib.collo_server_memory(self.h, C.byref(a), C.byref(pk)))
        return int(a.value), int(pk.value)

    def poll(self, ticket: int):
        problem, _ = self._keep[ticket]
        res = Result()
        theta = np.zeros(problem.p)
        res.theta = theta.ctypes.data
        st = lib.collo_server_poll(self.h, int(ticket), C.byref(res))
        if st == PENDING:
            return None
        _check(st)
        return _result_dict(res, theta, None, None)

    def close(self):
        if getattr(self, "h", None):
            lib.collo_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PROFILE_PHASES = ["eval", "rhs", "factor", "solve", "step", "linesearch", "update", "admit"]


def phase_profile(reset: bool = True):
    """collo_phase_profile: {phase: (ms, rounds)}, or None when COLLO_PROFILE is off."""
    ms = (C.c_double * 8)()
    rounds = (C.c_longlong * 8)()
    if lib.collo_phase_profile(ms, rounds, 8, int(reset)) == 0:
        return None
    return {k: (ms[i], rounds[i]) for i, k in enumerate(PROFILE_PHASES)}


def alu_peak(precision: int) -> float:
    """Measured FMA throughput (TFLOP/s) of the current device, FP64 or FP32."""
    t = C.c_double()
    _check(lib.collo_alu_peak(int(precision), C.byref(t)))
    return t.value


def launch_count() -> int:
    """Kernels launched by the library since load (collo_launch_count)."""
    return int(lib.collo_launch_count())


def version() -> str:
    return lib.collo_version().decode()
