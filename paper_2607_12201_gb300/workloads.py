"""Seeded synthetic parameter-estimation instances (inputs only).

This module draws the problem data that both the CUDA library and the CPU
oracle consume: a mass-action reaction network, its initial state, the
estimated-parameter set with bounds and a starting point, and noisy
observations of some species.  It contains none of the solution method's
arithmetic: no collocation, no derivatives, no linear algebra.  The
observations come from an independent ODE integrator (``scipy``'s LSODA, or
the closed form for the linear cascade), used here purely as a data source.

The problem statement being instantiated is Eq. 1 of the paper (an ODE
``dz/dt = f(z, theta)``, ``z(0) = x0``, parameters bounded,
least-squares misfit to measurements).  The workloads stand in for the
paper's PEtab systems-biology benchmark models (3-75 ODEs, 3-113 parameters,
Section "Selected benchmark models"), which are not available here.

Instance fields (all numpy, C-contiguous):

* ``n``, ``r``: species and reactions.
* ``react[r,2]``, ``prod[r,2]``: reactant / product species (-1 = unused
  slot; a repeated species means stoichiometry 2).
* ``pidx[r]``: index of the estimated parameter driving reaction r, or -1
  when the rate constant is fixed at ``kfix[r]``.
* ``logscale``: 1 if ``k = 10**theta`` (log10 parameters), 0 if
  ``k = theta``.
* ``x0[n]``; ``theta_true``, ``theta0``, ``theta_lo``, ``theta_hi`` (``[p]``).
* ``T``, ``N`` (uniform elements), ``K`` (collocation nodes per element).
* ``obs_t``, ``obs_s``, ``obs_y``, ``obs_sigma`` (``[M]``), sorted by time.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

LN10 = math.log(10.0)


@dataclasses.dataclass
class Instance:
    name: str
    seed: int
    n: int
    r: int
    react: np.ndarray
    prod: np.ndarray
    pidx: np.ndarray
    kfix: np.ndarray
    logscale: int
    x0: np.ndarray
    theta_true: np.ndarray
    theta0: np.ndarray
    theta_lo: np.ndarray
    theta_hi: np.ndarray
    T: float
    N: int
    K: int
    obs_t: np.ndarray
    obs_s: np.ndarray
    obs_y: np.ndarray
    obs_sigma: np.ndarray
    redraws: int = 0
    # collocation nodes: "radau" (right Radau, tau_K = 1) or "gauss" (Gauss-Legendre)
    scheme: str = "radau"
    # experimental conditions (Eq. 1d): each condition's initial state and its
    # inputs multiplying the rate constants, and the condition of each
    # measurement; None: one condition starting from x0.  N is the number of
    # elements of each condition's mesh.
    cond_x0: np.ndarray | None = None      # [Nc][n]
    cond_scale: np.ndarray | None = None   # [Nc][r]
    obs_cond: np.ndarray | None = None     # [M]

    @property
    def p(self) -> int:
        return int(self.theta_true.shape[0])

    @property
    def M(self) -> int:
        return int(self.obs_t.shape[0])

    @property
    def Nc(self) -> int:
        return 1 if self.cond_x0 is None else int(np.asarray(self.cond_x0).shape[0])

    @property
    def n_x(self) -> int:
        return self.n * self.N * self.Nc * (self.K + 1) + self.p

    @property
    def n_c(self) -> int:
        return self.n * self.N * self.Nc * (self.K + 1)

    def with_mesh(self, N: int) -> "Instance":
        return dataclasses.replace(self, N=int(N))

    def with_theta0(self, theta0) -> "Instance":
        return dataclasses.replace(self, theta0=np.ascontiguousarray(theta0, dtype=np.float64))


def _rng(*key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(list(key))))


def _rate_constants(react, pidx, kfix, logscale, theta):
    k = np.array(kfix, dtype=np.float64, copy=True)
    est = pidx >= 0
    th = theta[pidx[est]]
    k[est] = np.power(10.0, th) if logscale else th
    return k


def _simulate(inst_fields, theta, times, scale=None):
    """Integrate the mass-action ODE with scipy (data source only); scale [r]
    multiplies the rate constants (an experimental condition's inputs)."""
    from scipy.integrate import solve_ivp

    react, prod, pidx, kfix, logscale, x0, T = inst_fields
    k = _rate_constants(react, pidx, kfix, logscale, theta)
    if scale is not None:
        k = k * scale
    n = x0.shape[0]
    r = react.shape[0]
    stoich = np.zeros((n, r))
    for j in range(r):
        for s in react[j]:
            if s >= 0:
                stoich[s, j] -= 1.0
        for s in prod[j]:
            if s >= 0:
                stoich[s, j] += 1.0

    def rhs(_t, x):
        v = k.copy()
        for slot in range(2):
            sl = react[:, slot]
            m = sl >= 0
            v[m] *= x[sl[m]]
        return stoich @ v

    def jac(_t, x):
        J = np.zeros((n, n))
        for j in range(r):
            a, b = react[j]
            if b < 0:
                J[:, a] += stoich[:, j] * k[j]
            else:
                J[:, a] += stoich[:, j] * k[j] * x[b]
                J[:, b] += stoich[:, j] * k[j] * x[a]
        return J

    sol = solve_ivp(rhs, (0.0, T), x0, method="LSODA", t_eval=times, rtol=1e-10,
                    atol=1e-12, jac=jac)
    if not sol.success or sol.y.shape[1] != len(times):
        return None
    return sol.y.T  # [len(times), n]


def _observations(times, species, traj, rng, mode):
    """Noisy measurements; returns arrays sorted by (time, species).

    ``additive``: y = x + 0.01 eps, sigma = 0.01.  ``multiplicative``:
    y = x (1 + 0.05 eps), sigma = 0.05 max(|y|, 0.1 max_t |y_s|, 1e-6), i.e. a
    5 % error model floored at 10 % of the species' largest measurement so that
    near-zero readings do not dominate the misfit (and at 1e-6 for a species
    that decays to nothing over the horizon).
    """
    t_list, s_list, y_list, sig_list = [], [], [], []
    ys = {}
    if mode != "additive":
        for s in species:
            ys[s] = traj[:, s] * (1.0 + 0.05 * rng.standard_normal(len(times)))
    for ti, t in enumerate(times):
        for s in species:
            x = traj[ti, s]
            if mode == "additive":
                y = x + 0.01 * rng.standard_normal()
                sig = 0.01
            else:
                y = ys[s][ti]
                sig = 0.05 * max(abs(y), 0.1 * np.max(np.abs(ys[s])), 1e-6)
            t_list.append(t)
            s_list.append(s)
            y_list.append(y)
            sig_list.append(sig)
    return (np.array(t_list), np.array(s_list, dtype=np.int32), np.array(y_list),
            np.array(sig_list))


def linear_cascade(N: int = 50, T: float = 10.0, seed: int = 1001, noise: bool = True,
                   theta_true=(0.7, 0.3), theta0=(1.0, 1.0), M: int = 20) -> Instance:
    """Two-state linear cascade x1' = -t1 x1, x2' = t1 x1 - t2 x2, x(0) = (1, 0).

    Reactions: x1 -> x2 (rate t1) and x2 -> nothing (rate t2), linear scale.
    ``M`` observations of x2 at t_m = m T / M with additive N(0, 0.01^2) noise.
    """
    rng = _rng(seed)
    th = np.array(theta_true, dtype=np.float64)
    times = np.array([m * T / M for m in range(1, M + 1)])
    a, b = th
    # closed-form trajectory (data source)
    x2 = a / (b - a) * (np.exp(-a * times) - np.exp(-b * times))
    traj = np.zeros((M, 2))
    traj[:, 0] = np.exp(-a * times)
    traj[:, 1] = x2
    if noise:
        ot, os_, oy, osig = _observations(times, [1], traj, rng, "additive")
    else:
        ot, os_, oy = times.copy(), np.ones(M, dtype=np.int32), x2.copy()
        osig = np.full(M, 0.01)
    return Instance(
        name=f"cascade_N{N}", seed=seed, n=2, r=2,
        react=np.array([[0, -1], [1, -1]], dtype=np.int32),
        prod=np.array([[1, -1], [-1, -1]], dtype=np.int32),
        pidx=np.array([0, 1], dtype=np.int32), kfix=np.zeros(2), logscale=0,
        x0=np.array([1.0, 0.0]), theta_true=th, theta0=np.array(theta0, dtype=np.float64),
        theta_lo=np.full(2, 1e-3), theta_hi=np.full(2, 1e2), T=float(T), N=int(N), K=3,
        obs_t=ot, obs_s=os_, obs_y=oy, obs_sigma=osig)


def random_network(n: int, r: int, *, log10k=(-2.0, 1.0), n_obs: int = 4, M: int = 50,
                   T: float = 20.0, N: int = 400, seed: int = 1002, est: str = "all",
                   theta0_spread: float = 0.5, max_redraw: int = 200,
                   name: str | None = None) -> Instance:
    """Random mass-action network (1-2 reactants, 1-2 products per reaction).

    ``est``: "all" estimates every log10 rate constant; "even" estimates the
    even-indexed reactions and fixes the others at their true values.
    ``theta0 = theta_true + U[-spread, spread]`` (log10 units).  Networks whose
    true trajectory leaves [0, 1e3] or fails to integrate are redrawn with the
    next seed; the number of redraws is recorded.
    """
    for attempt in range(max_redraw):
        rng = _rng(seed, attempt)
        react = -np.ones((r, 2), dtype=np.int32)
        prod = -np.ones((r, 2), dtype=np.int32)
        for j in range(r):
            while True:
                nr = int(rng.integers(1, 3))
                npd = int(rng.integers(1, 3))
                rs = np.sort(rng.integers(0, n, size=nr))
                ps = np.sort(rng.integers(0, n, size=npd))
                if not (nr == npd and np.array_equal(rs, ps)):
                    break
            react[j, :nr] = rs
            prod[j, :npd] = ps
        lk = rng.uniform(log10k[0], log10k[1], size=r)
        x0 = rng.uniform(0.1, 1.0, size=n)
        if est == "all":
            pidx = np.arange(r, dtype=np.int32)
        else:
            pidx = -np.ones(r, dtype=np.int32)
            pidx[0::2] = np.arange((r + 1) // 2, dtype=np.int32)
        p = int(pidx.max()) + 1
        theta_true = np.zeros(p)
        kfix = np.power(10.0, lk)
        for j in range(r):
            if pidx[j] >= 0:
                theta_true[pidx[j]] = lk[j]
                kfix[j] = 0.0
        times = np.array([m * T / M for m in range(1, M + 1)])
        fields = (react, prod, pidx, kfix, 1, x0, T)
        dense_t = np.linspace(0.0, T, 401)
        traj_dense = _simulate(fields, theta_true, dense_t)
        if traj_dense is None or not np.all(np.isfinite(traj_dense)):
            continue
        if traj_dense.max() > 1e3 or traj_dense.min() < -1e-6:
            continue
        traj = _simulate(fields, theta_true, times)
        if traj is None:
            continue
        species = np.sort(rng.choice(n, size=n_obs, replace=False))
        ot, os_, oy, osig = _observations(times, species, traj, rng, "multiplicative")
        theta0 = theta_true + rng.uniform(-theta0_spread, theta0_spread, size=p)
        return Instance(
            name=name or f"massaction_n{n}_r{r}_N{N}", seed=seed, n=n, r=r, react=react,
            prod=prod, pidx=pidx, kfix=kfix, logscale=1, x0=x0, theta_true=theta_true,
            theta0=theta0, theta_lo=np.full(p, -5.0), theta_hi=np.full(p, 5.0), T=float(T),
            N=int(N), K=3, obs_t=ot, obs_s=os_, obs_y=oy, obs_sigma=osig, redraws=attempt)
    raise RuntimeError("no admissible network drawn")


# --- the five workloads (sizes of the paper-shaped configurations) ---------

def config1(**kw) -> Instance:
    """Linear cascade, Radau K=3, N=50, T=10, 20 noisy x2 observations."""
    return linear_cascade(**kw)


def config2(seed: int = 3, N: int = 400, theta0_spread: float = 0.1) -> Instance:
    """10 species / 20 reactions, log10 k ~ U[-2,1], 4 observed x 50 times, T=20."""
    return random_network(10, 20, log10k=(-2.0, 1.0), n_obs=4, M=50, T=20.0, N=N,
                          seed=seed, theta0_spread=theta0_spread,
                          name=f"massaction_n10_r20_N{N}")


def multistart_thetas(inst: Instance, count: int, seed: int = 2002,
                      spread: float = 0.1) -> list:
    """Seeded starting points theta_true + U[-spread, spread] (log10 units) for
    a multistart run of one instance."""
    rng = _rng(seed, 31337)
    return [inst.theta_true + rng.uniform(-spread, spread, inst.p) for _ in range(count)]


def config3(seed: int = 1003, N: int = 2000, est: str = "even",
            theta0_spread: float = 0.1) -> Instance:
    """Stiff: 30 species / 60 reactions, log10 k ~ U[-3,3], 8 observed x 100 times, T=50."""
    return random_network(30, 60, log10k=(-3.0, 3.0), n_obs=8, M=100, T=50.0, N=N,
                          seed=seed, est=est, theta0_spread=theta0_spread,
                          name=f"stiff_n30_r60_N{N}")


def multistart_batch(count: int = 256, seed: int = 1004, n_range=(5, 50),
                     N_range=(100, 2000), M: int = 50, T: float = 20.0) -> list[Instance]:
    """Uneven multistart batch: n ~ U{5..50}, r = 2n, N log-uniform, theta0 within +-1 decade."""
    out = []
    for j in range(count):
        rng = _rng(seed, 7919, j)
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        N = int(round(math.exp(rng.uniform(math.log(N_range[0]), math.log(N_range[1])))))
        inst = random_network(n, 2 * n, log10k=(-2.0, 1.0), n_obs=min(4, n), M=M, T=T, N=N,
                              seed=seed * 100003 + j, theta0_spread=1.0,
                              name=f"multistart{j}_n{n}_N{N}")
        out.append(inst)
    return out


def serving_stream(count: int = 64, seed: int = 1005, rate_hz: float = 200.0,
                   n_range=(5, 100), N_range=(200, 5000), M: int = 50, T: float = 20.0):
    """Poisson request stream: (arrival time, instance) with n, N log-uniform."""
    rng = _rng(seed, 104729)
    t = 0.0
    out = []
    for j in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        N = int(round(math.exp(rng.uniform(math.log(N_range[0]), math.log(N_range[1])))))
        inst = random_network(n, 2 * n, log10k=(-2.0, 1.0), n_obs=min(4, n), M=M, T=T, N=N,
                              seed=seed * 100003 + j, theta0_spread=0.5,
                              name=f"request{j}_n{n}_N{N}")
        out.append((t, inst))
    return out


def multi_condition(n: int = 6, r: int = 12, Nc: int = 3, N: int = 30, M: int = 20,
                    T: float = 10.0, seed: int = 1006, theta0_spread: float = 0.1,
                    n_inputs: int = 2, max_redraw: int = 50) -> Instance:
    """A random mass-action network measured under Nc experimental conditions
    (Eq. 1d): condition 0 is the network's own draw; every other condition has
    its own initial state x0^c ~ U[0.1, 1] and scales n_inputs of the rate
    constants by 10^U[-0.7, 0.7] (the condition-dependent inputs p^c of Eq. 3,
    lifted to multipliers of the rate constants).  Each condition is simulated
    and measured like the single network (same observed species and times,
    5 % multiplicative noise); the measurements are concatenated with their
    condition index."""
    base = random_network(n, r, n_obs=min(4, n), M=M, T=T, N=N, seed=seed,
                          theta0_spread=theta0_spread, name=f"conditions{Nc}_n{n}_r{r}_N{N}")
    species = np.unique(base.obs_s)
    times = np.array([m * T / M for m in range(1, M + 1)])
    fields = (base.react, base.prod, base.pidx, base.kfix, 1, base.x0, T)
    for attempt in range(max_redraw):
        rng = _rng(seed, 271828, attempt)
        x0s = [base.x0] + [rng.uniform(0.1, 1.0, size=n) for _ in range(Nc - 1)]
        scale = np.ones((Nc, r))
        for c in range(1, Nc):
            for j in rng.choice(r, size=min(n_inputs, r), replace=False):
                scale[c, j] = 10.0 ** rng.uniform(-0.7, 0.7)
        ts, ss, ys, sg, oc = [], [], [], [], []
        ok = True
        for c in range(Nc):
            fc = fields[:5] + (x0s[c], T)
            dense = _simulate(fc, base.theta_true, np.linspace(0.0, T, 201), scale[c])
            traj = _simulate(fc, base.theta_true, times, scale[c])
            if (dense is None or traj is None or not np.all(np.isfinite(dense))
                    or dense.max() > 1e3 or dense.min() < -1e-6):
                ok = False
                break
            t_, s_, y_, g_ = _observations(times, species, traj, rng, "multiplicative")
            ts.append(t_); ss.append(s_); ys.append(y_); sg.append(g_)
            oc.append(np.full(len(t_), c, dtype=np.int32))
        if not ok:
            continue
        return dataclasses.replace(
            base, obs_t=np.concatenate(ts), obs_s=np.concatenate(ss), obs_y=np.concatenate(ys),
            obs_sigma=np.concatenate(sg), cond_x0=np.array(x0s), cond_scale=scale,
            obs_cond=np.concatenate(oc), redraws=base.redraws + attempt)
    raise RuntimeError("no admissible conditions drawn")


def small_network(n: int = 3, r: int = 4, N: int = 4, seed: int = 7, M: int = 6,
                  T: float = 2.0, n_obs: int | None = None) -> Instance:
    """Tiny random network for brute-force checks."""
    return random_network(n, r, log10k=(-1.0, 0.5), n_obs=n_obs or min(2, n), M=M, T=T,
                          N=N, seed=seed, name=f"tiny_n{n}_r{r}_N{N}")
