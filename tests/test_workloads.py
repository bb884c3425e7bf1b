"""The seeded input generators follow the stated recipes (CPU): sizes,
distributions, the 5 % noise model with its floor, the estimated-parameter
selection, and determinism under a fixed seed."""
import numpy as np

from paper_2607_12201_gb300 import workloads as W


def _check_network(inst, n, r, M_per_species, T, log10k, spread):
    assert (inst.n, inst.r, inst.T, inst.K, inst.logscale) == (n, r, T, 3, 1)
    for j in range(r):
        rs = sorted(int(s) for s in inst.react[j] if s >= 0)
        ps = sorted(int(s) for s in inst.prod[j] if s >= 0)
        assert 1 <= len(rs) <= 2 and 1 <= len(ps) <= 2 and rs != ps
    lk = np.where(inst.pidx >= 0, np.nan, np.log10(np.maximum(inst.kfix, 1e-300)))
    est = inst.theta_true
    assert np.all((est >= log10k[0]) & (est <= log10k[1]))
    fixed = lk[~np.isnan(lk)]
    assert np.all((fixed >= log10k[0] - 1e-12) & (fixed <= log10k[1] + 1e-12))
    assert np.all((inst.x0 >= 0.1) & (inst.x0 <= 1.0))
    assert np.all(np.abs(inst.theta0 - inst.theta_true) <= spread)
    assert np.all(inst.theta_lo == -5.0) and np.all(inst.theta_hi == 5.0)
    species = np.unique(inst.obs_s)
    times = np.unique(inst.obs_t)
    assert len(times) == M_per_species and inst.M == len(species) * M_per_species
    assert np.allclose(times, np.arange(1, M_per_species + 1) * T / M_per_species)
    for s in species:                       # sigma = 0.05 max(|y|, 0.1 max_t |y_s|, 1e-6)
        sel = inst.obs_s == s
        ys = inst.obs_y[sel]
        floor = max(0.1 * np.max(np.abs(ys)), 1e-6)
        assert np.allclose(inst.obs_sigma[sel], 0.05 * np.maximum(np.abs(ys), floor), rtol=1e-14)


def test_config2_recipe():
    inst = W.config2()
    _check_network(inst, 10, 20, 50, 20.0, (-2.0, 1.0), 0.1)
    assert inst.N == 400 and inst.p == 20 and len(np.unique(inst.obs_s)) == 4


def test_config3_estimates_the_even_indexed_reactions():
    inst = W.config3(N=40)
    _check_network(inst, 30, 60, 100, 50.0, (-3.0, 3.0), 0.1)
    assert inst.p == 30
    assert np.array_equal(inst.pidx[0::2], np.arange(30)) and np.all(inst.pidx[1::2] == -1)
    assert np.all(inst.kfix[0::2] == 0.0) and np.all(inst.kfix[1::2] > 0.0)


def test_cascade_recipe():
    inst = W.config1()
    assert (inst.n, inst.N, inst.T, inst.M) == (2, 50, 10.0, 20)
    assert np.allclose(inst.obs_t, 0.5 * np.arange(1, 21)) and np.all(inst.obs_s == 1)
    assert np.all(inst.obs_sigma == 0.01) and np.array_equal(inst.theta0, [1.0, 1.0])


def test_multistart_batch_and_serving_stream_recipes():
    for inst in W.multistart_batch(count=6):
        assert 5 <= inst.n <= 50 and inst.r == 2 * inst.n and 100 <= inst.N <= 2000
        assert np.all(np.abs(inst.theta0 - inst.theta_true) <= 1.0)
    stream = W.serving_stream(count=40)
    arrivals = np.array([a for a, _ in stream])
    assert np.all(np.diff(arrivals) > 0)
    assert 1.0 / 400 < arrivals[-1] / len(arrivals) < 1.0 / 100      # mean gap near 1/200 s
    for _, inst in stream:
        assert 5 <= inst.n <= 100 and inst.r == 2 * inst.n and 200 <= inst.N <= 5000


def test_generators_are_deterministic():
    a, b = W.config2(), W.config2()
    for f in ("react", "prod", "theta_true", "theta0", "x0", "obs_t", "obs_y", "obs_sigma"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    s1 = W.multistart_thetas(a, 4, seed=2002)
    s2 = W.multistart_thetas(b, 4, seed=2002)
    assert all(np.array_equal(u, v) for u, v in zip(s1, s2))
