#!/usr/bin/env python
"""Benchmark of the GPU Radau-collocation interior-point path.

Workload: the 10-species / 20-reaction random mass-action network on
N = 400 Radau elements (K = 3), 4 observed species x 50 times, T = 20,
seed 3 (``workloads.config2()``): 16 020 primal unknowns, 16 000 constraints,
20 log10 rate constants, solved from Q seeded starting points
theta_true + U[-0.1, 0.1] (a multistart run; ``--queue``, default 256).

A timed step serves the Q starts through the continuous-batching server
(``collo_server_*``) with ``--slots`` (default 64) slots: all Q are submitted
at once, admitted as slots free up (in groups of ``--admit``), and every
server step advances all admitted solves by one Newton step in batched
launches, in the mixed-precision path (FP32 element factorization and block
cyclic reduction, FP64 parameter Schur complement, residuals and refinement,
FP64 factorization where refinement from FP32 fails).  ``value`` = Newton steps per second over
all Q solves.  Beside it: one lock-step batch of ``--slots`` starts (no
refill), the same path and the plain FP64 path on a single instance,
per-solve latency percentiles, the parameter agreement with FP64 solves, an
end-to-end number through host buffers, the dominant kernel's roofline and
the CPU oracle.  Between timed steps the L2 cache is flushed (256 MiB write).

``--impl reference`` times the CPU oracle instead (a bounded sample: each step
is the oracle's initial point plus two Newton iterations of one instance).

Multi-GPU (torchrun, one process per GPU): each rank serves its own queue
with no collective on the data path (weak scaling); the timed region is
bracketed by barriers and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = ("massaction_n10_r20_N400_K3 x {Q} multistart solves served with {S} slots "
            "(config 2: 10 species, 20 reactions, N=400, T=20, seed 3; "
            "starts theta_true + U[-0.1,0.1])")
METRIC = "Newton steps/s (mixed-precision continuous-batching IPM path, config 2 multistart)"
# KKT tolerance of every solve in the benchmark: at the paper's 1e-6 the mixed
# and FP64 paths stop at points up to 4e-3 apart in rate constants along flat
# directions of the objective (same iterations, same objective to 1e-12); at
# 1e-8 they agree within the 1e-6 parameter criterion.
TOL = 1e-8
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one
# element-condensation launch over 64 config-2 instances, from an ncu capture
# of that launch (--only-elem-phase --slots 64); None once the kernel changes.
ELEM_TRAFFIC_S64 = 1.0576e9


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the reduced uneven-batch and Poisson-stream measurements")
    ap.add_argument("--batch", type=int, default=64,
                    help="instances of --only-batch")
    ap.add_argument("--slots", type=int, default=64)
    ap.add_argument("--queue", type=int, default=256)
    ap.add_argument("--admit", type=int, default=32,
                    help="admit waiting solves in groups of at least this many free slots")
    ap.add_argument("--only-solve", choices=["mixed", "fp64"], default=None,
                    help="run one single-instance solve and exit (for profiler launch lists)")
    ap.add_argument("--only-batch", action="store_true",
                    help="run one batched solve and exit (for profiler launch lists)")
    ap.add_argument("--only-elem-phase", action="store_true",
                    help="evaluate --slots config-2 problems at their forward-sweep states and "
                         "launch the batched element condensation twice (ncu capture)")
    ap.add_argument("--phase-profile", action="store_true",
                    help="serve the queue twice with the driver's phase profile on and print it")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def reduce_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "samples": len(sm),
                "reasons": sorted(reasons)}


def _pair_flops(msz: int, pairs: int) -> int:
    """Flops of eliminating `pairs` 2x2 pivots from a symmetric msz x msz block:
    pair q updates t(t+1)/2 trailing entries with two FMAs and forms 2t
    multipliers with four FMAs per row (t = msz - 2q - 2)."""
    fl = 0
    for q in range(pairs):
        t = msz - 2 * q - 2
        fl += 2 * t * (t + 1) + 8 * t
    return fl


def elem_factor_work(n: int, p: int, N: int, bytes_per: int):
    """Algorithmic flops and bytes of one element-condensation launch.

    Per element: eliminating the 3n interior pairs of the symmetric (8n + p)
    block.  Bytes: FP64 derivative blocks read (jac_z, hess_zz at 3 n^2,
    jac_theta, hess_ztheta at 3 n p, objective block 16 n doubles) and the
    factor written (6n L columns of length 8n + p, 3n pivots, the 2n x 2n
    interface block, its 2n x p border, the p x p FP64 Schur part)."""
    ext = 8 * n + p
    fl = _pair_flops(ext, 3 * n)
    rd = 8 * (2 * 3 * n * n + 2 * 3 * n * p + 16 * n)
    wr = bytes_per * (6 * n * ext + 9 * n + 4 * n * n + n * n + 2 * n * p) + 8 * p * p
    return fl * N, (rd + wr) * N


def factor_work(n: int, p: int, N: int, bytes_per: int):
    """Algorithmic flops and bytes of one whole factorization of one instance:
    element condensation (above), the N eliminations of the cyclic reduction
    (n pairs of a (4n + p) block each: interface block, neighbour couplings
    and border read, L columns written), the parameter Schur complement
    (2N p^2 FP64 contributions summed, p^3/3 for its LDL^T)."""
    fl_e, by_e = elem_factor_work(n, p, N, bytes_per)
    bext = 4 * n + p
    fl_b = _pair_flops(bext, n) * N
    by_b = bytes_per * N * (4 * n * n + 2 * n * n + 2 * n * p + 2 * n * bext + 3 * n)
    fl_s = p ** 3 // 3 + 2 * N * p * p
    by_s = 8 * 2 * N * p * p
    return fl_e + fl_b + fl_s, by_e + by_b + by_s


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def rate_rel_err(theta, theta_ref):
    """Largest relative error of the rate constants k = 10**theta."""
    import numpy as np
    return float(np.max(np.abs(np.expm1(np.log(10.0) * (np.asarray(theta) - theta_ref)))))


def run_ours(args):
    import numpy as np
    import torch

    from paper_2607_12201_gb300 import build as B
    B.build()
    from paper_2607_12201_gb300 import collo, workloads

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    init_dist(world, "nccl")
    inst = workloads.config2()
    S, Q = args.slots, args.queue
    starts = workloads.multistart_thetas(inst, Q, seed=2002 + rank)
    probs = [collo.Problem(inst, device=local) for _ in range(Q)]
    server = collo.Server(S, device=local, precision=collo.MIXED, tol=TOL)
    server.set_admission(args.admit)
    sstream = torch.cuda.ExternalStream(server.stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def flush_l2(i):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()

    def timed_serve():
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(sstream)
        tickets = [server.submit(p, theta0=th) for p, th in zip(probs, starts)]
        while True:
            act, wait = server.step()
            if act == 0 and wait == 0:
                break
        e1.record(sstream)
        e1.synchronize()
        return [server.poll(t) for t in tickets], e0.elapsed_time(e1)

    for i in range(args.warmup):
        flush_l2(i)
        timed_serve()
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = collo.launch_count()
    its, ms_list, statuses, lat, last = 0, [], [], [], None
    for i in range(args.steps):
        flush_l2(i)
        res, ms = timed_serve()
        its += sum(r["iterations"] for r in res)
        ms_list.append(ms)
        statuses += [r["status"] for r in res]
        lat += [1e3 * r["wall"] for r in res]
        last = res
    launches = collo.launch_count() - l0
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    t_total = reduce_max(sum(ms_list), world)
    its_total = reduce_sum(float(its), world)
    solves_total = reduce_sum(float(args.steps * Q), world)
    conv_total = reduce_sum(float(sum(1 for s_ in statuses if s_ in (collo.OK, collo.ACCEPTABLE))),
                            world)
    value = its_total / (t_total * 1e-3)

    # one lock-step batch of S starts (no refill), on the problems' own streams
    bstream = torch.cuda.ExternalStream(probs[0].stream)
    flush_l2(0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(bstream)
    bres = collo.batch_solve(probs[:S], theta0s=starts[:S], precision=collo.MIXED, tol=TOL)
    e1.record(bstream)
    e1.synchronize()
    b_ms = e0.elapsed_time(e1)
    b_its = sum(r["iterations"] for r in bres)

    # single-instance paths on the same GPU: mixed and the plain FP64 path
    one = probs[0]
    single = {}
    for name, prec in [("mixed", collo.MIXED), ("fp64", collo.FP64)]:
        one.ipm_solve(theta0=starts[0], precision=prec, want_x=False, tol=TOL)
        ms_s, its_s = [], 0
        for i in range(3):
            flush_l2(i)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(bstream)
            r = one.ipm_solve(theta0=starts[0], precision=prec, want_x=False, tol=TOL)
            e1.record(bstream)
            e1.synchronize()
            ms_s.append(e0.elapsed_time(e1))
            its_s += r["iterations"]
        single[name] = {"newton_steps_per_s": its_s / (sum(ms_s) * 1e-3),
                        "solves_per_s": len(ms_s) / (sum(ms_s) * 1e-3),
                        "ms_per_solve": sum(ms_s) / len(ms_s)}
    # parameter agreement of the served mixed solves with single FP64 solves
    perr, n_cmp = 0.0, 0
    for j in range(min(8, Q)):
        if last[j]["status"] not in (collo.OK, collo.ACCEPTABLE):
            continue
        r64 = one.ipm_solve(theta0=starts[j], precision=collo.FP64, want_x=False, tol=TOL)
        if r64["status"] in (collo.OK, collo.ACCEPTABLE):
            perr = max(perr, rate_rel_err(last[j]["theta"], r64["theta"]))
            n_cmp += 1

    # phase timings at S instances (CUDA events inside the library)
    ph = {"factor_fp32": collo.batch_time_phase(probs[:S], 1, collo.MIXED, reps=5),
          "factor_fp32_elements": collo.batch_time_phase(probs[:S], 4, collo.MIXED, reps=5),
          "factor_fp32_reduction_schur": collo.batch_time_phase(probs[:S], 5, collo.MIXED, reps=5),
          "solve_fp32": collo.batch_time_phase(probs[:S], 2, collo.MIXED, reps=5),
          "eval": collo.batch_time_phase(probs[:S], 3, collo.MIXED, reps=5)}
    peak32 = collo.alu_peak(collo.MIXED)
    peak64 = collo.alu_peak(collo.FP64)
    # dominant kernel: the FP32 element condensation (FP32 FMA bound)
    fl_e, by_e = elem_factor_work(inst.n, inst.p, inst.N, 4)
    fl_e *= S
    by_e *= S
    ach = fl_e / (ph["factor_fp32_elements"] * 1e-3) / 1e12
    # ALU peak from the unit counts and the clock: SMs x 128 FP32 lanes x 2 flops
    # (FMA) x maximum SM clock
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = clk.get("sm_max_mhz") or 2070.0
    peak_alu = sms * 128 * 2 * mhz * 1e6 / 1e12
    roof = {"bound": "alu", "achieved": ach, "peak": peak_alu, "unit": "TFLOP/s",
            "frac": ach / peak_alu,
            "traffic": ELEM_TRAFFIC_S64 * S / 64 if ELEM_TRAFFIC_S64 else None,
            "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 flops x {mhz:.0f} MHz; measured "
                           f"FFMA throughput {peak32:.1f} TFLOP/s (collo_alu_peak)",
            "kernel": f"k_elem_factor_rt_b<float> (element condensation, {S} instances)",
            "algorithmic_flops": fl_e, "algorithmic_bytes": by_e,
            "ms": ph["factor_fp32_elements"],
            "hbm": {"achieved_gbs": by_e / (ph["factor_fp32_elements"] * 1e-3) / 1e9,
                    "peak_gbs": measured_peaks().get("hbm_gbs")}}

    out = {
        "metric": METRIC, "value": value, "unit": "Newton steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp32 factor + fp64 residual/refinement",
        "data": "synthetic (seeded mass-action network, noisy observations, seeded starts)",
        "config": {"workload": WORKLOAD.format(Q=Q, S=S), "queue": Q, "slots": S, "tol": TOL,
                   "admit_group": args.admit,
                   "step": f"serve {Q} starts from theta0 to a final status",
                   "newton_steps_per_step": its / max(args.steps, 1),
                   "n_x_per_instance": one.n_x, "n_c_per_instance": one.n_c, "p": inst.p,
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{world} (independent queues)"},
        "solves_per_s": solves_total / (t_total * 1e-3),
        "converged_solves_per_s": conv_total / (t_total * 1e-3),
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "what": "per-solve service time, admission to final status"},
        "status_counts": {str(s_): statuses.count(s_) for s_ in sorted(set(statuses))},
        "lockstep_batch": {"instances": S, "newton_steps_per_s": b_its / (b_ms * 1e-3),
                           "ms": b_ms, "what": f"one collo_batch_solve of {S} starts, no refill"},
        "single_instance": single,
        "speedup_vs_fp64_single": value / single["fp64"]["newton_steps_per_s"],
        "solves_speedup_vs_fp64_single": (solves_total / (t_total * 1e-3))
                                         / single["fp64"]["solves_per_s"],
        "param_rel_err_vs_fp64": {"value": perr, "compared": n_cmp,
                                  "what": "max |k_mixed/k_fp64 - 1| over rate constants "
                                          "k = 10^theta, starts where both paths converged"},
        "phases_ms": ph, "roofline": roof,
        "peaks_tflops": {"fp32_ffma": peak32, "fp64_dfma": peak64},
        "gpu_launches": launches, "clocks": clk,
    }
    if not args.no_e2e:
        keep = [inst.react, inst.prod, inst.pidx, inst.kfix, inst.x0, inst.theta_lo,
                inst.theta_hi, inst.obs_t, inst.obs_s, inst.obs_y, inst.obs_sigma]
        h2d = Q * int(sum(np.asarray(a).nbytes for a in keep)) + 8 * inst.p * Q
        tot, its_e = 0.0, 0
        k_e = max(1, min(args.steps, 2))
        for i in range(k_e):
            flush_l2(i)
            t0 = time.perf_counter()
            ps = [collo.Problem(inst, device=local) for _ in range(Q)]
            tk = [server.submit(p, theta0=th) for p, th in zip(ps, starts)]
            while True:
                act, wait = server.step()
                if act == 0 and wait == 0:
                    break
            res = [server.poll(t) for t in tk]
            for pb in ps:
                pb.close()
            t1 = time.perf_counter()
            tot += t1 - t0
            its_e += sum(r["iterations"] for r in res)
        tot = reduce_max(tot, world)
        its_e = reduce_sum(float(its_e), world)
        out["e2e"] = {"value": its_e / tot, "unit": "Newton steps/s",
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": Q * (8 * inst.p + 64),
                      "what": f"{Q} x collo_problem_create from host arrays + serving + "
                              "theta* read back, per step", "steps": k_e}
    if not args.no_extra:
        out.update(uneven_and_stream(collo, workloads, local))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(inst, iters=6)
    if rank == 0:
        print(json.dumps(out), flush=True)
    server.close()
    for pb in probs:
        pb.close()


def uneven_and_stream(collo, workloads, device):
    """Reduced-size versions of the uneven multistart batch and the Poisson
    serving stream (species 5-15, 100-800 elements): mixed path through the
    server, against the plain FP64 path solving the same instances one by one."""
    import numpy as np
    out = {}
    # uneven batch: all submitted at once, served through 16 slots
    insts = workloads.multistart_batch(count=48, n_range=(5, 15), N_range=(100, 400))
    probs = [collo.Problem(i, device=device) for i in insts]
    srv = collo.Server(16, device=device, precision=collo.MIXED, tol=TOL)
    srv.set_admission(4)
    for rep in range(2):   # the first pass allocates the factor storage
        t0 = time.perf_counter()
        tk = [srv.submit(p) for p in probs]
        while True:
            act, wait = srv.step()
            if act == 0 and wait == 0:
                break
        dt = time.perf_counter() - t0
        res = [srv.poll(t) for t in tk]
    srv.close()
    t64 = 0.0
    for p in probs:
        t1 = time.perf_counter()
        p.ipm_solve(precision=collo.FP64, want_x=False, tol=TOL)
        t64 += time.perf_counter() - t1
    lat = [1e3 * r["wall"] for r in res]
    out["uneven_batch"] = {
        "instances": len(probs), "slots": 16, "species": [5, 15], "elements": [100, 400],
        "sizes_n_N": [[i.n, i.N] for i in insts],
        "newton_steps_per_s": sum(r["iterations"] for r in res) / dt,
        "solves_per_s": len(res) / dt,
        "fp64_single_solves_per_s": len(probs) / t64,
        "solves_speedup_vs_fp64_single": (len(res) / dt) / (len(probs) / t64),
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "status_counts": {str(s_): sum(1 for r in res if r["status"] == s_)
                          for s_ in sorted(set(r["status"] for r in res))},
        "what": "config-4 shape at reduced sizes, served through 16 slots (admission groups "
                "of 4); fp64 single = the same instances solved one after another on the plain "
                "FP64 path"}
    for p in probs:
        p.close()
    # Poisson stream: requests submitted at their arrival times (host clock)
    stream = workloads.serving_stream(count=48, rate_hz=200.0, n_range=(5, 15),
                                      N_range=(200, 800))
    probs = [collo.Problem(i, device=device) for _, i in stream]
    srv = collo.Server(64, device=device, precision=collo.MIXED, tol=TOL)
    srv.set_admission(1)
    for rep in range(2):
        t0 = time.perf_counter()
        nxt, tk, done_at = 0, {}, {}
        while len(done_at) < len(stream):
            now = time.perf_counter() - t0
            while nxt < len(stream) and stream[nxt][0] <= now:
                tk[nxt] = srv.submit(probs[nxt])
                nxt += 1
            act, wait = srv.step()
            for j, t in tk.items():
                if j not in done_at and srv.poll(t) is not None:
                    done_at[j] = time.perf_counter() - t0
            if act == 0 and wait == 0 and nxt < len(stream):
                time.sleep(max(0.0, stream[nxt][0] - (time.perf_counter() - t0)))
        dt = time.perf_counter() - t0
        res = [srv.poll(tk[j]) for j in range(len(stream))]
    srv.close()
    lat = [1e3 * (done_at[j] - stream[j][0]) for j in range(len(stream))]
    out["poisson_stream"] = {
        "requests": len(stream), "rate_hz": 200.0, "species": [5, 15], "elements": [200, 800],
        "newton_steps_per_s": sum(r["iterations"] for r in res) / dt,
        "solves_per_s": len(res) / dt,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "status_counts": {str(s_): sum(1 for r in res if r["status"] == s_)
                          for s_ in sorted(set(r["status"] for r in res))},
        "what": "config-5 shape at reduced sizes: seeded exponential gaps, each request "
                "submitted at its arrival time; latency = arrival to result (host clock)"}
    for p in probs:
        p.close()
    return out


def cpu_baseline(inst, iters):
    from oracle import ipm as oipm
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    t0 = time.perf_counter()
    r = oipm.solve(inst, opt=oipm.Options(max_iter=iters))
    dt = time.perf_counter() - t0
    return {"value": r.iterations / dt, "unit": "Newton steps/s", "cores": cores,
            "kind": "oracle",
            "sample": f"oracle IPM on the same config-2 instance: initial point + {r.iterations} "
                      f"Newton iterations ({dt:.1f} s, numpy/scipy FP64, block KKT mode)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1:
        init_dist(world, "gloo")
        if rank != 0:
            return
    from oracle import ipm as oipm
    from paper_2607_12201_gb300 import workloads
    inst = workloads.config2()
    inst = inst.with_theta0(workloads.multistart_thetas(inst, 1, seed=2002)[0])
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    per = 2
    for _ in range(args.warmup):
        oipm.solve(inst, opt=oipm.Options(max_iter=per))
    t0 = time.perf_counter()
    its = 0
    for _ in range(args.steps):
        its += oipm.solve(inst, opt=oipm.Options(max_iter=per)).iterations
    dt = time.perf_counter() - t0
    v = its / dt
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Newton steps/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "fp64", "data": "synthetic",
           "config": {"workload": WORKLOAD.format(Q=args.queue, S=args.slots),
                      "step": f"oracle initial point + {per} Newton iterations of one start"},
           "cpu_baseline": {"value": v, "unit": "Newton steps/s", "cores": cores,
                            "kind": "oracle",
                            "sample": f"{args.steps} x (initial point + {per} Newton iterations)"},
           "e2e": {"value": v, "unit": "Newton steps/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def only_solve(prec_name):
    from paper_2607_12201_gb300 import build as B
    B.build()
    from paper_2607_12201_gb300 import collo, workloads
    inst = workloads.config2()
    prec = collo.MIXED if prec_name == "mixed" else collo.FP64
    with collo.Problem(inst) as prob:
        l0 = collo.launch_count()
        r = prob.ipm_solve(precision=prec, want_x=False)
        print(json.dumps({"only_solve": prec_name, "status": r["status"],
                          "iterations": r["iterations"], "wall_s": r["wall"],
                          "launches": collo.launch_count() - l0}), flush=True)
        if r["status"] not in (collo.OK, collo.ACCEPTABLE):
            sys.exit(1)


def phase_profile(args):
    """Per-phase host wall time of the IPM driver while serving (COLLO_PROFILE=1:
    the driver synchronises at each phase boundary, so the total is a little
    above an unprofiled run)."""
    os.environ["COLLO_PROFILE"] = "1"
    from paper_2607_12201_gb300 import build as B
    B.build()
    from paper_2607_12201_gb300 import collo, workloads
    inst = workloads.config2()
    S, Q = args.slots, args.queue
    starts = workloads.multistart_thetas(inst, Q, seed=2002)
    probs = [collo.Problem(inst) for _ in range(Q)]
    server = collo.Server(S, precision=collo.MIXED, tol=TOL)
    server.set_admission(args.admit)
    for rep in range(2):
        collo.phase_profile(reset=True)
        t0 = time.perf_counter()
        tk = [server.submit(p, theta0=th) for p, th in zip(probs, starts)]
        n_steps = 0
        while True:
            act, wait = server.step()
            n_steps += 1
            if act == 0 and wait == 0:
                break
        wall = time.perf_counter() - t0
        res = [server.poll(t) for t in tk]
        prof = collo.phase_profile(reset=True)
    print(json.dumps({"phase_profile": {k: {"ms": round(v[0], 1), "rounds": v[1]}
                                        for k, v in prof.items()},
                      "wall_s": round(wall, 3), "server_steps": n_steps,
                      "newton_steps": sum(r["iterations"] for r in res),
                      "factorizations": sum(r["factorizations"] for r in res),
                      "fp64_factorizations": sum(r["fp64_facs"] for r in res),
                      "refinement_sweeps": sum(r["refine"] for r in res),
                      "line_search_trials": sum(r["trials"] for r in res),
                      "queue": Q, "slots": S, "admit_group": args.admit, "tol": TOL}), flush=True)
    server.close()


def only_elem_phase(S):
    from paper_2607_12201_gb300 import build as B
    B.build()
    from paper_2607_12201_gb300 import collo, workloads
    inst = workloads.config2()
    starts = workloads.multistart_thetas(inst, S, seed=2002)
    probs = [collo.Problem(inst) for _ in range(S)]
    for p, th in zip(probs, starts):
        x, _ = p.initial_states(th)
        p.eval_raw(x.ctypes.data, None)
    ms = collo.batch_time_phase(probs, 4, collo.MIXED, reps=1)
    print(json.dumps({"only_elem_phase": S, "elements": S * inst.N, "ms": ms}), flush=True)
    for p in probs:
        p.close()


def only_batch(nb):
    from paper_2607_12201_gb300 import build as B
    B.build()
    from paper_2607_12201_gb300 import collo, workloads
    inst = workloads.config2()
    starts = workloads.multistart_thetas(inst, nb, seed=2002)
    probs = [collo.Problem(inst) for _ in range(nb)]
    l0 = collo.launch_count()
    t0 = time.perf_counter()
    res = collo.batch_solve(probs, theta0s=starts, precision=collo.MIXED)
    print(json.dumps({"only_batch": nb, "wall_s": time.perf_counter() - t0,
                      "iterations": sum(r["iterations"] for r in res),
                      "status": sorted(set(r["status"] for r in res)),
                      "launches": collo.launch_count() - l0}), flush=True)
    for pb in probs:
        pb.close()


def main():
    args = parse_args()
    if args.only_solve:
        only_solve(args.only_solve)
    elif args.only_batch:
        only_batch(args.batch)
    elif args.phase_profile:
        phase_profile(args)
    elif args.only_elem_phase:
        only_elem_phase(args.slots)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
