"""Batched solves and continuous batching: each problem's result is the same
alone and in a mix (bitwise: every kernel computes an instance from its own
data in a fixed order), and batched results match the oracle."""
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


def _mix():
    return [W.config1(),
            W.random_network(4, 8, n_obs=3, M=20, T=5.0, N=40, seed=41, theta0_spread=0.1),
            W.small_network(n=3, r=4, N=7, seed=7),
            W.config2(N=100),
            W.random_network(12, 24, n_obs=4, M=20, T=5.0, N=33, seed=43, theta0_spread=0.1)]


def _mixed_paths():
    # element blocks of 8n + p = 50 (register tiles), 130 (shared memory) and, in
    # FP64, 150 rows (216.8 KB: factored in a global slab) in one batch
    return [W.random_network(5, 10, n_obs=3, M=20, T=5.0, N=24, seed=51, theta0_spread=0.1),
            W.random_network(13, 26, n_obs=4, M=20, T=5.0, N=20, seed=52, theta0_spread=0.1),
            W.random_network(15, 30, n_obs=4, M=20, T=5.0, N=18, seed=53, theta0_spread=0.1)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_mixed_factor_paths_equals_alone(collo, prec):
    P = collo.MIXED if prec == "mixed" else collo.FP64
    insts = _mixed_paths()
    alone = []
    for inst in insts:
        with collo.Problem(inst) as pb:
            alone.append(pb.ipm_solve(precision=P, want_x=False, max_iter=12))
    probs = [collo.Problem(inst) for inst in insts]
    mixed = collo.batch_solve(probs, precision=P, max_iter=12)
    for a, b in zip(alone, mixed):
        assert a["status"] == b["status"]
        assert a["iterations"] == b["iterations"]
        assert np.array_equal(a["theta"], b["theta"])
    for pb in probs:
        pb.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_equals_alone_bitwise(collo, prec):
    P = collo.MIXED if prec == "mixed" else collo.FP64
    insts = _mix()
    alone = []
    for inst in insts:
        with collo.Problem(inst) as pb:
            alone.append(pb.ipm_solve(precision=P, want_x=False))
    probs = [collo.Problem(inst) for inst in insts]
    mixed = collo.batch_solve(probs, precision=P)
    for a, b in zip(alone, mixed):
        assert a["status"] == b["status"]
        assert a["iterations"] == b["iterations"]
        assert np.array_equal(a["theta"], b["theta"])
        assert a["phi"] == b["phi"]
    for pb in probs:
        pb.close()


def test_full_size_batch_equals_alone_bitwise(collo):
    # 6 x 400 elements: the first reduction level has more blocks (1200) than the
    # persistent factor kernel has block halves, so a half factors several blocks
    # of a level and stages the next one's inputs during the current elimination;
    # the solve runs its levels 0-4 over the grid and the rest per instance.  The
    # same starts alone never overlap two blocks.  Iterates must be bitwise equal.
    inst = W.config2()
    starts = W.multistart_thetas(inst, 6, seed=2002)
    alone = []
    for th in starts:
        with collo.Problem(inst) as pb:
            alone.append(pb.ipm_solve(theta0=th, precision=collo.MIXED, max_iter=6))
    probs = [collo.Problem(inst) for _ in starts]
    mixed = collo.batch_solve(probs, theta0s=starts, precision=collo.MIXED, max_iter=6,
                              want_x=True)
    for a, b in zip(alone, mixed):
        assert a["iterations"] == b["iterations"]
        assert a["factorizations"] == b["factorizations"]
        assert np.array_equal(a["theta"], b["theta"])
        assert np.array_equal(a["x"], b["x"])
        assert np.array_equal(a["lam"], b["lam"])
    for pb in probs:
        pb.close()


def test_batch_multistart_matches_oracle(collo):
    base = W.random_network(4, 8, n_obs=3, M=20, T=5.0, N=40, seed=41, theta0_spread=0.1)
    rng = np.random.default_rng(5)
    starts = [base.theta_true + rng.uniform(-0.2, 0.2, base.p) for _ in range(4)]
    probs = [collo.Problem(base) for _ in starts]
    res = collo.batch_solve(probs, theta0s=starts, precision=collo.MIXED)
    for r, th0 in zip(res, starts):
        ref = oipm.solve(base.with_theta0(th0))
        assert r["status"] == ref.status
        if ref.status in (0, 1):
            rel = np.max(np.abs(r["theta"] - ref.x[-base.p:]) / np.abs(ref.x[-base.p:]))
            assert rel <= 1e-6
    for pb in probs:
        pb.close()


def test_server_continuous_batching_equals_alone(collo):
    insts = _mix()
    alone = []
    for inst in insts:
        with collo.Problem(inst) as pb:
            alone.append(pb.ipm_solve(precision=collo.MIXED, want_x=False))
    server = collo.Server(max_slots=3, precision=collo.MIXED)
    probs = [collo.Problem(inst) for inst in insts]
    tickets = {}
    # staggered arrivals: one new request every other step, 3 slots
    step = 0
    pending = list(range(len(insts)))
    done = {}
    while len(done) < len(insts):
        if pending and step % 2 == 0:
            i = pending.pop(0)
            tickets[i] = server.submit(probs[i])
        server.step()
        for i, t in tickets.items():
            if i not in done:
                r = server.poll(t)
                if r is not None:
                    done[i] = r
        step += 1
        assert step < 5000
    for i, a in enumerate(alone):
        b = done[i]
        assert a["status"] == b["status"]
        assert a["iterations"] == b["iterations"]
        assert np.array_equal(a["theta"], b["theta"])
    server.close()
    for pb in probs:
        pb.close()


def test_repeated_batches_are_bitwise_reproducible(collo):
    insts = _mix()
    runs = []
    for _ in range(3):
        probs = [collo.Problem(inst) for inst in insts]
        runs.append(collo.batch_solve(probs, precision=collo.MIXED))
        for pb in probs:
            pb.close()
    for r in runs[1:]:
        for a, b in zip(runs[0], r):
            assert a["iterations"] == b["iterations"]
            assert np.array_equal(a["theta"], b["theta"])


def test_server_admits_by_device_memory_budget(collo):
    """Admission by device memory: with a budget of k problems' full footprint
    (their arrays plus the factorization stores a mixed-precision solve
    allocates, collo_problem_solve_bytes) at most k of n waiting problems run at
    once although more slots are free; the held memory never exceeds the budget;
    each job's stores are freed when it retires; every result equals the same
    problem solved alone."""
    inst = W.random_network(4, 8, n_obs=3, M=20, T=5.0, N=40, seed=41, theta0_spread=0.1)
    rng = np.random.default_rng(11)
    starts = [inst.theta_true + rng.uniform(-0.1, 0.1, inst.p) for _ in range(6)]
    probs = [collo.Problem(inst) for _ in starts]
    need = probs[0].solve_bytes(collo.MIXED)
    base = probs[0].device_bytes()
    assert need > base          # the stores are counted before they exist
    k = 2
    budget = k * need + need // 2
    server = collo.Server(max_slots=5, budget_bytes=budget, precision=collo.MIXED)
    tickets = [server.submit(pb, th) for pb, th in zip(probs, starts)]
    most, done = 0, {}
    for _ in range(5000):
        active, waiting = server.step()
        held, peak = server.memory()
        most = max(most, active)
        assert active <= k and held <= budget and peak <= budget
        for i, t in enumerate(tickets):
            if i not in done:
                r = server.poll(t)
                if r is not None:
                    done[i] = r
                    # retired: its factorization stores are freed (its arrays,
                    # the spare trial arrays included, stay with the problem)
                    assert base <= probs[i].device_bytes() < need
                    assert probs[i].solve_bytes(collo.MIXED) == need
        if len(done) == len(tickets):
            break
    assert most == k
    assert server.memory()[1] == k * need
    server.close()
    for i, (pb, th) in enumerate(zip(probs, starts)):
        alone = pb.ipm_solve(theta0=th, precision=collo.MIXED, want_x=False)
        assert alone["status"] == done[i]["status"]
        assert alone["iterations"] == done[i]["iterations"]
        assert np.array_equal(alone["theta"], done[i]["theta"])
        pb.close()


def test_server_fails_a_problem_larger_than_the_budget(collo):
    inst = W.small_network(n=3, r=4, N=7, seed=7)
    small = collo.Problem(inst)
    big = collo.Problem(W.config2(N=100))
    budget = small.solve_bytes(collo.FP64) + 1024
    assert big.solve_bytes(collo.FP64) > budget
    server = collo.Server(max_slots=2, budget_bytes=budget)
    t_big = server.submit(big)
    t_small = server.submit(small)
    for _ in range(2000):
        server.step()
        if server.poll(t_small) is not None:
            break
    assert server.poll(t_big)["status"] == collo.ERR_OOM
    assert server.poll(t_small)["status"] in (collo.OK, collo.ACCEPTABLE)
    server.close()
    small.close()
    big.close()


def test_autotuner_picks_a_schedule_and_results_stay_correct(collo, tmp_path):
    """collo_autotune times the large-element kernel and the solve under each
    candidate schedule on an uneven batch, keeps the fastest (no slower than the
    schedule it started from), and caches it; solves under the tuned schedule
    are bitwise reproducible and agree with the default schedule's within the
    parity tolerance (the panel width changes the rounding of slab blocks)."""
    insts = [W.random_network(n, 2 * n, n_obs=4, M=20, T=5.0, N=N, seed=70 + n,
                              theta0_spread=0.1) for n, N in ((6, 40), (20, 30), (36, 20))]
    default = collo.get_schedule()
    probs = [collo.Problem(i) for i in insts]
    ref = collo.batch_solve(probs, precision=collo.MIXED, max_iter=8)
    try:
        cache = str(tmp_path / "sched.json")
        best, before, after, hit = collo.autotune(probs, collo.MIXED, reps=2, cache=cache)
        assert not hit and after <= before
        assert best == collo.get_schedule()
        again = collo.autotune(probs, collo.MIXED, reps=2, cache=cache)
        assert again[3] and again[0] == best
        runs = [collo.batch_solve(probs, precision=collo.MIXED, max_iter=8) for _ in range(2)]
        for a, b, r in zip(runs[0], runs[1], ref):
            assert np.array_equal(a["theta"], b["theta"])
            assert a["iterations"] == r["iterations"]
            assert np.max(np.abs(a["theta"] - r["theta"])) <= 1e-6 * max(1.0, np.max(np.abs(r["theta"])))
    finally:
        collo.set_schedule(default)
        for pb in probs:
            pb.close()
