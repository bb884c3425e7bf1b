#!/usr/bin/env python
"""Benchmark of the GPU Radau-collocation interior-point path.

Workload (the uneven multistart batch at its stated size,
``workloads.multistart_batch()``): 256 seeded mass-action networks, species
n ~ U{5..50}, reactions r = 2n (all rate constants estimated, p = 2n),
N log-uniform on [100, 2000] Radau elements (K = 3), 4 observed species x 50
times, T = 20, starts theta0 within +-1 decade of the true log10 rate
constants: 40.2 M KKT unknowns in all, 157 k per instance on average.

The instances are served through the continuous-batching server
(``collo_server_*``) with ``--slots`` slots (default 64) inside a device-memory
budget (default 180 GiB), in the mixed-precision path (FP32 element and
cyclic-reduction factors, FP64 parameter Schur complement, residuals and
refinement, FP64 factorization where refinement from FP32 fails), every solve
to KKT tolerance 1e-8.  Every instance that reaches a final status is
submitted again from the same start, so the server runs a steady multistart
stream.  One benchmark step is ``--slice`` server steps (default 8), each
advancing every admitted solve by one Newton step in batched launches;
``value`` = Newton steps per second over all solves.  Beside it: solves that
reached a final status per second (all, and converged), their service-time
percentiles, the plain FP64 single-instance path on a stratified subsample of
the same instances, the parameter agreement of converged served solves with
FP64 solves of the same starts, per-kernel timings and rooflines, an
end-to-end number through host buffers, the config-2 multistart workload (on
Radau and on Gauss-Legendre K = 4 points), a Poisson stream of the
serving-stream shape, and the CPU oracle.

``--impl reference`` times the CPU oracle instead (a bounded sample: each step
is the oracle's initial point plus two Newton iterations of one instance of
the batch).

Multi-GPU (torchrun, one process per GPU): each rank serves its own copy of
the stream with no collective on the data path (weak scaling); the timed
region is bracketed by barriers and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

# the oracle (cpu_baseline and the reference arm) makes thousands of small
# LAPACK calls; one BLAS thread is its fastest setting here
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = ("uneven multistart batch at its stated size: 256 mass-action networks, "
            "n ~ U{{5..50}} species, r = p = 2n, N log-uniform [100, 2000], K = 3, "
            "4 observed x 50 times, T = 20, starts within +-1 decade (seed 1004); served "
            "as a steady multistart stream (finished instances resubmitted) through {S} "
            "slots within a {B} GiB device-memory budget")
METRIC = ("Newton steps/s (mixed-precision continuous-batching IPM path, uneven multistart "
          "batch at its stated size)")
# KKT tolerance of every solve in the benchmark: at the paper's 1e-6 the mixed
# and FP64 paths stop at points up to 4e-3 apart in rate constants along flat
# directions of the objective (same iterations, same objective to 1e-12); at
# 1e-8 they agree within the 1e-6 parameter criterion.
TOL = 1e-8
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a
# kernel over the first 64 instances of the batch at their initial points,
# from one ncu capture of that launch (--only-phase); None until captured or
# once the kernel changes.
TRAFFIC_C4_64 = {"elem_big": 6077422592 + 15532304896,
                 "reduction_schur": 5363395072 + 4618892288,
                 "solve": 18268539648 + 184806400}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--slots", type=int, default=64)
    ap.add_argument("--slice", type=int, default=8, help="server steps per benchmark step")
    ap.add_argument("--admit", type=int, default=32,
                    help="admit waiting solves in groups of at least this many free slots")
    ap.add_argument("--budget-gib", type=float, default=180.0)
    ap.add_argument("--fp64-sample", type=int, default=8,
                    help="instances of the stratified subsample run on the plain FP64 path")
    ap.add_argument("--fp64-steps", type=int, default=20,
                    help="Newton steps of each FP64 single-instance run")
    ap.add_argument("--no-tune", action="store_true", help="keep the default schedule")
    ap.add_argument("--schedule-cache", default=None,
                    help="JSON file caching autotuned schedules per batch shape and device")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the config-2 multistart and Poisson-stream measurements")
    ap.add_argument("--only-phase", type=int, default=0,
                    help="time one batched phase (1..7 of collo_batch_time_phase) over the "
                         "first --slots instances at their initial points and exit (ncu)")
    ap.add_argument("--phase-case", default="batch", choices=["batch", "large"],
                    help="--only-phase instances: the first --slots of the batch, or --slots "
                         "copies of one 45-species network on N = 150 (element blocks of 450 "
                         "rows, factored in the global slab)")
    ap.add_argument("--only-serve", type=int, default=0,
                    help="run this many server steps of the stream and exit (ncu launch list)")
    ap.add_argument("--only-next", action="store_true",
                    help="run the conditions batch and the refinement loop and exit")
    ap.add_argument("--only-lifted", action="store_true",
                    help="run the lifted vs augmented step comparison and exit")
    ap.add_argument("--lifted-case", default="both", choices=["both", "config2", "config3"],
                    help="--only-lifted: which configuration")
    ap.add_argument("--phase-profile", action="store_true",
                    help="print the driver's per-phase wall time over --slice server steps")
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


def _pair_l_entries(msz: int, pairs: int) -> int:
    """Entries of the L columns of `pairs` eliminated 2x2 pivots (rows below each pair)."""
    return sum(2 * (msz - 2 * q - 2) for q in range(pairs))


def elem_factor_work(n: int, p: int, N: int, bytes_per: int):
    """Algorithmic flops and bytes of the element condensation of one instance.

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


def reduction_work(n: int, p: int, N: int, bytes_per: int):
    """Algorithmic flops and bytes of the cyclic reduction and the parameter
    Schur complement of one instance: N eliminations of n pairs of a (4n + p)
    block (interface block, two couplings and border read, L columns and pivots
    written, the neighbours' blocks and borders updated), the 2N p^2 FP64
    contributions summed and the p^3 / 3 of the Schur block's LDL^T."""
    bext = 4 * n + p
    fl = _pair_flops(bext, n) * N + p ** 3 // 3 + 2 * N * p * p
    by = bytes_per * N * (4 * n * n + 2 * n * n + 2 * n * p + 2 * n * bext + 3 * n
                          + 2 * (n * n + n * p)) + 8 * 2 * N * p * p
    return fl, by


def solve_bytes(n: int, p: int, N: int, bytes_per: int):
    """Algorithmic bytes of one solve (no refinement): the used entries of the
    element and reduction L columns and their pivots read twice (forward and
    back substitution), the right-hand side read and the solution written in
    FP64, the per-block intermediate vectors written and read once."""
    ext, bext = 8 * n + p, 4 * n + p
    lent = N * (_pair_l_entries(ext, 3 * n) + _pair_l_entries(bext, n))
    piv = N * 3 * (3 * n + n)
    nk = 8 * n * N + p
    inter = N * (6 * n + 2 * n + 2 * n)
    return 2 * bytes_per * (lent + piv) + 8 * 2 * nk + 2 * bytes_per * inter


def eval_bytes(n: int, p: int, N: int):
    """Algorithmic bytes of one evaluation with derivatives: x and lambda read,
    constraints, gradient, the Jacobian and Hessian blocks (3 n^2 and 3 n p per
    element each, 16 n objective entries) and per-element partial sums written."""
    nk = 8 * n * N + p
    return 8 * (nk + N * (2 * 3 * n * n + 2 * 3 * n * p + 16 * n + 4 + p))


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def rate_rel_err(theta, theta_ref):
    """Largest relative error of the rate constants k = 10**theta."""
    import numpy as np
    return float(np.max(np.abs(np.expm1(np.log(10.0) * (np.asarray(theta) - theta_ref)))))


class Stream:
    """A steady multistart stream through a server: every instance that
    reaches a final status is submitted again from the same start.  With
    `recreate` each resubmission first builds a new problem from the
    instance's host arrays (and frees the finished one), the end-to-end form."""

    def __init__(self, collo, server, insts, probs, device):
        self.collo, self.server, self.insts, self.probs = collo, server, insts, probs
        self.device = device
        self.recreate = False
        self.h2d = 0
        self.d2h = 0
        self.tk = {server.submit(p): i for i, p in enumerate(probs)}

    def step(self, m):
        """m server steps; the (instance, result) pairs that finished in them."""
        fin = []
        for _ in range(m):
            self.server.step()
            for t in list(self.tk):
                r = self.server.poll(t)
                if r is None:
                    continue
                i = self.tk.pop(t)
                fin.append((i, r))
                self.d2h += 8 * self.insts[i].p
                if self.recreate:
                    self.probs[i].close()
                    self.probs[i] = self.collo.Problem(self.insts[i], device=self.device)
                    self.h2d += host_bytes(self.insts[i])
                self.tk[self.server.submit(self.probs[i])] = i
        return fin


def host_bytes(inst):
    """Bytes of an instance's host arrays that collo_problem_create copies to the device."""
    import numpy as np
    keep = [inst.react, inst.prod, inst.pidx, inst.kfix, inst.x0, inst.theta_lo, inst.theta_hi,
            inst.obs_t, inst.obs_s, inst.obs_y, inst.obs_sigma, inst.theta0]
    return int(sum(np.asarray(a).nbytes for a in keep))


def stratified(insts, k):
    """k instances spread over the batch by the work of one factorization
    (N (8n + p)^3): the middles of k equal strata of the sorted list."""
    order = sorted(range(len(insts)), key=lambda i: insts[i].N * (8 * insts[i].n + insts[i].p) ** 3)
    return [order[int((j + 0.5) * len(order) / k)] for j in range(k)]


def run_ours(args):
    import numpy as np
    import torch

    from paper_2607_12201_gb300 import build as B
    B.build()
    from paper_2607_12201_gb300 import collo, workloads

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    init_dist(world, "nccl")
    S, M = args.slots, args.slice
    budget = int(args.budget_gib * (1 << 30))
    insts = workloads.multistart_batch()
    tune = autotune_schedule(collo, insts[:S], local, args) if not args.no_tune else None
    probs = [collo.Problem(i, device=local) for i in insts]
    server = collo.Server(S, budget_bytes=budget, device=local, precision=collo.MIXED, tol=TOL)
    server.set_admission(args.admit)
    sstream = torch.cuda.ExternalStream(server.stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    st = Stream(collo, server, insts, probs, local)

    def timed_slice(i):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        c0 = server.counters()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(sstream)
        fin = st.step(M)
        e1.record(sstream)
        e1.synchronize()
        c1 = server.counters()
        return e0.elapsed_time(e1), [b - a for a, b in zip(c0, c1)], fin

    warm_fin = []
    for i in range(args.warmup):
        warm_fin += timed_slice(i)[2]
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = collo.launch_count()
    ms_list, its, done, conv, fin_all = [], 0, 0, 0, []
    for i in range(args.steps):
        ms, d, fin = timed_slice(i)
        ms_list.append(ms)
        its += d[0]
        done += d[1]
        conv += d[2]
        fin_all += fin
    launches = collo.launch_count() - l0
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    t_total = reduce_max(sum(ms_list), world)
    its_total = reduce_sum(float(its), world)
    done_total = reduce_sum(float(done), world)
    conv_total = reduce_sum(float(conv), world)
    value = its_total / (t_total * 1e-3)
    held, peak = server.memory()
    statuses = [r["status"] for _, r in fin_all]
    lat = [1e3 * r["wall"] for _, r in fin_all]
    its_fin = sum(r["iterations"] for _, r in fin_all) or 1
    per_step = {"factorizations": sum(r["factorizations"] for _, r in fin_all) / its_fin,
                "fp64_factorizations": sum(r["fp64_facs"] for _, r in fin_all) / its_fin,
                "solves": 1.0 + sum(r["refine"] for _, r in fin_all) / its_fin,
                "evaluations": 1.0 + sum(r["trials"] for _, r in fin_all) / its_fin}

    out = {
        "metric": METRIC, "value": value, "unit": "Newton steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp32 factor + fp64 residual/refinement",
        "data": "synthetic (seeded mass-action networks, noisy observations, seeded starts)",
        "config": {"workload": WORKLOAD.format(S=S, B=args.budget_gib), "instances": len(insts),
                   "kkt_unknowns_total": int(sum(8 * i.n * i.N + i.p for i in insts)),
                   "slots": S, "budget_gib": args.budget_gib, "tol": TOL,
                   "admit_group": args.admit,
                   "step": f"{M} server steps of the steady stream (each advances every "
                           "admitted solve by one Newton step)",
                   "newton_steps_per_step": its / max(args.steps, 1),
                   "l2": "inputs larger than L2 (factor stores of tens of GB per step); "
                         "also flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{world} (independent streams)"},
        "solves_per_s": done_total / (t_total * 1e-3),
        "converged_solves_per_s": conv_total / (t_total * 1e-3),
        "latency_ms": {"p50": float(np.percentile(lat, 50)) if lat else None,
                       "p99": float(np.percentile(lat, 99)) if lat else None,
                       "count": len(lat),
                       "what": "service time (admission to final status) of the solves "
                               "that finished in the timed steps"},
        "status_counts": {str(s_): statuses.count(s_) for s_ in sorted(set(statuses))},
        "per_newton_step": per_step,
        "autotune": tune,
        "memory_gib": {"held_at_end": held / 2 ** 30, "peak": peak / 2 ** 30},
        "gpu_launches": launches, "clocks": clk,
    }

    # end to end through host buffers: the same stream, each resubmission a new
    # problem created from the instance's host arrays, every result read back
    if not args.no_e2e:
        st.recreate = True
        st.h2d = st.d2h = 0
        k_e = max(1, min(args.steps, 2))
        torch.cuda.synchronize()
        c0 = server.counters()
        t0 = time.perf_counter()
        for i in range(k_e):
            st.step(M)
        torch.cuda.synchronize()
        dt = reduce_max(time.perf_counter() - t0, world)
        c1 = server.counters()
        out["e2e"] = {"value": reduce_sum(float(c1[0] - c0[0]), world) / dt,
                      "unit": "Newton steps/s",
                      "h2d_bytes_per_step": st.h2d / k_e, "d2h_bytes_per_step": st.d2h / k_e,
                      "what": "the same stream, host clock; every resubmitted instance is a new "
                              "collo_problem_create from host arrays (the finished problem is "
                              "destroyed) and every result's theta is read back",
                      "steps": k_e}
    server.close()
    for pb in st.probs:
        pb.close()
    del probs

    # the plain FP64 single-instance path on a stratified subsample
    sample = stratified(insts, args.fp64_sample)
    ms64, its64 = 0.0, 0
    for i in sample:
        with collo.Problem(insts[i], device=local) as pb:
            pst = torch.cuda.ExternalStream(pb.stream)
            pb.ipm_solve(precision=collo.FP64, want_x=False, tol=TOL, max_iter=1)   # allocation
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(pst)
            r = pb.ipm_solve(precision=collo.FP64, want_x=False, tol=TOL,
                             max_iter=args.fp64_steps)
            e1.record(pst)
            e1.synchronize()
            ms64 += e0.elapsed_time(e1)
            its64 += r["iterations"]
    fp64_rate = its64 / (ms64 * 1e-3)
    mean_its = its_fin / max(len(fin_all), 1)
    out["fp64_single"] = {
        "newton_steps_per_s": fp64_rate,
        "solves_per_s_derived": fp64_rate / mean_its,
        "instances": [[insts[i].n, insts[i].N] for i in sample],
        "what": f"plain FP64 path, one instance at a time (collo_ipm_solve), on a stratified "
                f"subsample of {len(sample)} instances (middles of equal strata of the batch "
                f"sorted by factorization work), first {args.fp64_steps} Newton steps of each; "
                "solves/s derived with the served solves' mean Newton steps per solve "
                f"({mean_its:.1f})"}
    out["speedup_vs_fp64_single"] = value / fp64_rate
    out["solves_speedup_vs_fp64_single"] = (done_total / (t_total * 1e-3)) / (fp64_rate / mean_its)

    # parameter agreement: converged served solves against FP64 solves of the same start
    perr, n_cmp = 0.0, 0
    seen = set()
    for i, r in warm_fin + fin_all:
        if r["status"] not in (collo.OK, collo.ACCEPTABLE) or i in seen or n_cmp >= 6:
            continue
        seen.add(i)
        with collo.Problem(insts[i], device=local) as pb:
            r64 = pb.ipm_solve(precision=collo.FP64, want_x=False, tol=TOL, max_wall_time=60.0)
        if r64["status"] in (collo.OK, collo.ACCEPTABLE):
            perr = max(perr, rate_rel_err(r["theta"], r64["theta"]))
            n_cmp += 1
    out["param_rel_err_vs_fp64"] = {
        "value": perr if n_cmp else None, "compared": n_cmp,
        "what": "max |k_mixed/k_fp64 - 1| over rate constants k = 10^theta, served solves "
                "that converged (warm-up and timed steps) against FP64 single solves of the "
                "same instance and start"}

    # per-kernel timings (CUDA events inside the library) over the first S
    # instances at their initial points, and their rooflines
    out.update(kernel_rooflines(collo, insts[:S], local, per_step, clk))
    if not args.no_extra:
        out.update(guarded("config2_multistart", config2_multistart, collo, workloads, local))
        out.update(guarded("config2_multistart_gauss_k4", config2_multistart, collo, workloads,
                           local, "gauss"))
        out.update(guarded("poisson_stream", poisson_stream, collo, workloads, local, budget))
        out.update(guarded("lifted_vs_augmented", lifted_comparison, collo, workloads, local))
        out.update(guarded("conditions_and_refinement", conditions_and_refinement, collo,
                           workloads, local))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(insts)
    if rank == 0:
        print(json.dumps(out), flush=True)


def autotune_schedule(collo, insts, device, args):
    """The launch schedule for this workload: collo_autotune over the first
    --slots instances at their initial points (cached per batch shape and
    device in --schedule-cache)."""
    import torch
    probs = [collo.Problem(i, device=device) for i in insts]
    for p, i in zip(probs, insts):
        x, _ = p.initial_states(i.theta0)
        p.eval_raw(x.ctypes.data, None)
    name = torch.cuda.get_device_name(device)
    best, before, after, hit = collo.autotune(probs, collo.MIXED, reps=2,
                                              cache=args.schedule_cache, device_name=name)
    for p in probs:
        p.close()
    return {"schedule": best, "default_ms": before, "tuned_ms": after,
            "gain": before / after if after > 0 else None, "from_cache": hit,
            "what": "collo_autotune over the first instances at their initial points: the "
                    "large-element kernel (threads per block, pairs per panel of slab blocks) "
                    "and the solve (per-instance top levels, elements per block) timed per "
                    "candidate; ms = the two phases' time per launch under the default and "
                    "the tuned schedule"}


def kernel_rooflines(collo, insts, device, per_step, clk):
    import torch
    probs = [collo.Problem(i, device=device) for i in insts]
    for p, i in zip(probs, insts):
        x, _ = p.initial_states(i.theta0)
        p.eval_raw(x.ctypes.data, None)
    F = collo.MIXED
    ms = {"elem_big": collo.batch_time_phase(probs, 6, F, reps=3),
          "elem_rt": collo.batch_time_phase(probs, 7, F, reps=3),
          "reduction_schur": collo.batch_time_phase(probs, 5, F, reps=3),
          "solve": collo.batch_time_phase(probs, 2, F, reps=3),
          "eval": collo.batch_time_phase(probs, 3, F, reps=3)}
    for p in probs:
        p.close()
    big = [i for i in insts if 8 * i.n + i.p > 124]
    small = [i for i in insts if 8 * i.n + i.p <= 124]
    w = {"elem_big": sum(elem_factor_work(i.n, i.p, i.N, 4)[0] for i in big),
         "elem_rt": sum(elem_factor_work(i.n, i.p, i.N, 4)[0] for i in small),
         "reduction_schur": sum(reduction_work(i.n, i.p, i.N, 4)[0] for i in insts),
         "solve": sum(solve_bytes(i.n, i.p, i.N, 4) for i in insts),
         "eval": sum(eval_bytes(i.n, i.p, i.N) for i in insts)}
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    mhz = clk.get("sm_max_mhz") or 2070.0
    peak_alu = sms * 128 * 2 * mhz * 1e6 / 1e12
    peak_hbm = measured_peaks().get("hbm_gbs") or 6800.0
    kern = {"elem_big": "k_elem_factor_big_b<float>", "elem_rt": "k_elem_factor_rt_b<float>",
            "reduction_schur": "k_factor_b<float> (cyclic reduction + parameter Schur)",
            "solve": "k_solve_b<float>", "eval": "k_eval_b<1> + k_eval_reduce_b"}
    roofs = {}
    for k, t in ms.items():
        if t <= 0:
            continue
        if k in ("solve", "eval"):
            ach = w[k] / (t * 1e-3) / 1e9
            roofs[k] = {"bound": "hbm", "achieved": ach, "peak": peak_hbm, "unit": "GB/s",
                        "frac": ach / peak_hbm, "traffic": TRAFFIC_C4_64.get(k),
                        "algorithmic": w[k], "ms": t, "kernel": kern[k]}
        else:
            ach = w[k] / (t * 1e-3) / 1e12
            roofs[k] = {"bound": "alu", "achieved": ach, "peak": peak_alu, "unit": "TFLOP/s",
                        "frac": ach / peak_alu, "traffic": TRAFFIC_C4_64.get(k),
                        "algorithmic": w[k], "ms": t, "kernel": kern[k]}
    # time per Newton step of the batch: each factorization runs the three
    # factorization kernels, each solve round the solve, each evaluation the eval
    share = {k: ms[k] * per_step["factorizations"] for k in ("elem_big", "elem_rt",
                                                               "reduction_schur")}
    share["solve"] = ms["solve"] * per_step["solves"]
    share["eval"] = ms["eval"] * per_step["evaluations"]
    dom = max((k for k in share if k in roofs), key=lambda k: share[k])
    tot = sum(share.values()) or 1.0
    roof = dict(roofs[dom])
    roof["peak_source"] = (f"{sms} SMs x 128 FP32 lanes x 2 flops x {mhz:.0f} MHz"
                           if roof["bound"] == "alu" else "MEASURED_PEAKS.json hbm_gbs")
    roof["share_of_kernel_time"] = share[dom] / tot
    return {"roofline": roof,
            "kernels": {k: dict(roofs[k], share_of_kernel_time=share[k] / tot) for k in roofs},
            "kernels_what": f"CUDA-event time per batched launch over the first {len(insts)} "
                            "instances at their initial points (collo_batch_time_phase); share = "
                            "that time x launches per Newton step of the served stream"}


def config2_multistart(collo, workloads, device, scheme="radau"):
    """The config-2 multistart workload: 256 starts of one 10-species network,
    served; scheme "gauss" runs the same on Gauss-Legendre K = 4 points."""
    inst = workloads.config2()
    if scheme == "gauss":
        inst = dataclasses.replace(inst, K=4, scheme="gauss")
    starts = workloads.multistart_thetas(inst, 256, seed=2002)
    probs = [collo.Problem(inst, device=device) for _ in starts]
    srv = collo.Server(64, device=device, precision=collo.MIXED, tol=TOL)
    srv.set_admission(32)
    for rep in range(2):
        t0 = time.perf_counter()
        tk = [srv.submit(p, theta0=th) for p, th in zip(probs, starts)]
        while True:
            act, wait = srv.step()
            if act == 0 and wait == 0:
                break
        dt = time.perf_counter() - t0
        res = [srv.poll(t) for t in tk]
    srv.close()
    for p in probs:
        p.close()
    its = sum(r["iterations"] for r in res)
    conv = sum(1 for r in res if r["status"] in (collo.OK, collo.ACCEPTABLE))
    key = "config2_multistart" if scheme == "radau" else "config2_multistart_gauss_k4"
    return {key: {
        "newton_steps_per_s": its / dt, "solves_per_s": len(res) / dt,
        "converged_solves_per_s": conv / dt, "wall_s": dt,
        "what": "256 starts (theta_true + U[-0.1, 0.1]) of the 10-species / 20-reaction "
                "network on N = 400 served through 64 slots, host clock, second pass"
                + ("; Gauss-Legendre K = 4 collocation" if scheme == "gauss" else "")}}


LIFTED_R = 1e-8   # relaxation of the lifted form's equalities


def lifted_start(prob, inst, mu=0.1, r=LIFTED_R):
    """Inputs of the lifted step at the interior-point start, from the GPU's own
    forward sweep and evaluation: theta pushed 1e-2 into its bounds, slacks
    s = c(x0) pushed into [-r, r], unit bound duals, lambda = 0.  Returns
    (sigma_x, sigma_s, r_x, r_s, r_c, augmented rhs)."""
    import numpy as np
    lo, hi = np.asarray(inst.theta_lo, float), np.asarray(inst.theta_hi, float)
    push = lambda v, a, b: np.minimum(np.maximum(v, a + np.minimum(1e-2 * np.maximum(1, abs(a)),
                                                                    1e-2 * (b - a))),
                                      b - np.minimum(1e-2 * np.maximum(1, abs(b)), 1e-2 * (b - a)))
    th = push(np.asarray(inst.theta0, float), lo, hi)
    x, _ = prob.initial_states(th)
    ev = prob.eval(x, None)
    c, grad = ev["c"], ev["grad"]
    s = np.clip(c, -r + 2e-2 * r, r - 2e-2 * r)
    nz = prob.n_x - prob.p
    sl, su = th - lo, hi - th
    sx = np.zeros(prob.n_x)
    sx[nz:] = 1.0 / sl + 1.0 / su
    ss = 1.0 / (s + r) + 1.0 / (r - s)
    gphi = grad.copy()
    gphi[nz:] += -mu / sl + mu / su
    rx = -gphi
    rs = -(-mu / (s + r) + mu / (r - s))
    rc = -(c - s)
    return sx, ss, rx, rs, rc, np.concatenate([rx, -c])


def lifted_flops(n, p, N, K=3, gauss=False):
    """Algorithmic FP64 flops of the lifted element kernel: J^T diag(d) J as one
    symmetric rank-1 update per constraint row over the row's nonzeros (a
    collocation row: K other points, its node-block row of n, its p parameter
    entries; a continuity row: 2 or K + 2 entries), 2 flops per updated
    lower-triangle entry, plus the Cholesky of the K n interior columns (the
    trailing update, 2 flops per updated entry)."""
    kn, me = K * n, K * n + 2 * n + p
    nz_col = K + n + p
    nz_cont = K + 2 if gauss else 2
    rank1 = kn * nz_col * (nz_col + 1) + n * nz_cont * (nz_cont + 1)
    chol = sum((me - c - 1) * (me - c) for c in range(kn))
    return N * (rank1 + chol)


def lifted_comparison(collo, workloads, device, which="both"):
    """The lifted condensed-space step against the augmented step on the same
    iterate: config 2 (N = 400) and config 3 (N = 2000)."""
    peak64 = collo.alu_peak(collo.FP64)
    out = {}
    cases = []
    if which in ("both", "config2"):
        cases.append(("config2_N400", workloads.config2()))
    if which in ("both", "config3"):
        cases.append(("config3_N2000", workloads.config3()))
    for key, inst in cases:
        with collo.Problem(inst, device=device) as prob:
            sx, ss, rx, rs, rc, rhs = lifted_start(prob, inst)
            dw = 0.0
            while not prob.lifted_factor(sx, ss, dw):
                dw = 1e-4 if dw == 0.0 else 8.0 * dw
            t0 = time.perf_counter()
            dx, ds, dl, info = prob.lifted_solve(rx, rs, rc, refine_max=20, refine_tol=1e-12)
            solve_wall = time.perf_counter() - t0
            ms_elem = prob.time_phase(5, reps=5)
            ms_fac = prob.time_phase(6, reps=5)
            ms_sol = prob.time_phase(7, reps=5)
            aug = {}
            mu = 0.1
            for name, prec in (("fp64", collo.FP64), ("mixed", collo.MIXED)):
                prob.kkt_factor(sx, 0.0, 1e-8 * mu ** 0.25, precision=prec)
                _, ainfo = prob.kkt_solve(rhs, refine_max=20, refine_tol=1e-12)
                aug[name] = {"factor_ms": prob.time_phase(1, prec, reps=5),
                             "solve_ms": prob.time_phase(2, prec, reps=5),
                             "refinement_sweeps": ainfo["sweeps"]}
        ipm = {}
        if key == "config2_N400":
            with collo.Problem(inst, device=device) as prob:
                for name, fn in (("lifted", lambda: prob.lifted_ipm_solve(want_x=False)),
                                 ("augmented_fp64",
                                  lambda: prob.ipm_solve(want_x=False, precision=collo.FP64)),
                                 ("augmented_mixed",
                                  lambda: prob.ipm_solve(want_x=False, precision=collo.MIXED))):
                    t0 = time.perf_counter()
                    r = fn()
                    dt = time.perf_counter() - t0
                    ipm[name] = {"status": r["status"], "iterations": r["iterations"],
                                 "wall_s": dt, "newton_steps_per_s": r["iterations"] / dt}
        fl = lifted_flops(inst.n, inst.p, inst.N, inst.K, getattr(inst, "scheme", "") == "gauss")
        ach = fl / (ms_elem * 1e-3) / 1e12
        out[key] = {"lifted": {"factor_ms": ms_fac, "elem_kernel_ms": ms_elem,
                               "solve_once_ms": ms_sol, "refinement_sweeps": info["sweeps"],
                               "residual": info["residual"], "delta_w": dw,
                               "solve_with_refinement_wall_ms": 1e3 * solve_wall},
                    "augmented": aug,
                    **({"whole_solve_from_theta0": ipm} if ipm else {}),
                    "elem_roofline": {"bound": "alu", "achieved": ach, "peak": peak64,
                                      "unit": "TFLOP/s", "frac": ach / peak64,
                                      "algorithmic_flops": fl,
                                      "kernel": "k_lifted_elem (FP64)",
                                      "peak_source": "collo_alu_peak FP64 FMA probe"}}
    out["what"] = ("one Newton step at the interior-point start (slacks c(x0) in [-r, r], "
                   f"r = {LIFTED_R:g}): lifted condensed Cholesky path (FP64) vs the augmented "
                   "2x2-pivot path (FP64 and mixed), same problem and iterate; CUDA events "
                   "per phase (collo_time_phase 1/2 and 5/6/7)")
    return {"lifted_vs_augmented": out}


def conditions_and_refinement(collo, workloads, device):
    """Beside the headline: a batch of multistart solves of the three-condition
    network (chains cut at each condition's first element, theta shared), and
    the batched mesh-refinement loop over config-2 starts from N = 100."""
    out = {}
    inst = workloads.multi_condition()
    starts = workloads.multistart_thetas(inst, 32, seed=2003)
    probs = [collo.Problem(inst, device=device) for _ in starts]
    t0 = time.perf_counter()
    res = collo.batch_solve(probs, theta0s=starts, precision=collo.MIXED, tol=TOL)
    dt = time.perf_counter() - t0
    for p in probs:
        p.close()
    its = sum(r["iterations"] for r in res)
    conv = sum(1 for r in res if r["status"] in (collo.OK, collo.ACCEPTABLE))
    out["conditions_batch"] = {
        "newton_steps_per_s": its / dt, "converged_solves_per_s": conv / dt, "solves": len(res),
        "converged": conv, "wall_s": dt,
        "what": "32 starts (theta_true + U[-0.1, 0.1]) of a 6-species network measured under "
                "3 experimental conditions (N = 30 per condition), one batched solve (mixed)"}
    c2 = workloads.config2(N=100)
    starts = workloads.multistart_thetas(c2, 16, seed=2004)
    probs = [collo.Problem(c2, device=device) for _ in starts]
    t0 = time.perf_counter()
    res, finals, levels = collo.refine_solve(probs, theta0s=starts, defect_tol=1e-6,
                                             max_levels=2, precision=collo.MIXED, tol=TOL)
    dt = time.perf_counter() - t0
    fin_N = [f.N for f in finals]
    for f, p in zip(finals, probs):
        if f is not p:
            f.close()
    for p in probs:
        p.close()
    out["refinement_loop"] = {
        "wall_s": dt, "solves": len(res), "levels": levels, "final_N": fin_N,
        "converged": sum(1 for r in res if r["status"] in (collo.OK, collo.ACCEPTABLE)),
        "what": "16 config-2 starts from N = 100: batched solve, then every converged solve "
                "whose collocation defect exceeds 1e-6 re-solved on twice the elements, warm "
                "started, up to two levels (collo_refine_solve, mixed)"}
    return out


def guarded(name, fn, *a):
    """An extra measurement that cannot take the benchmark line down with it."""
    try:
        return fn(*a)
    except Exception as e:   # reported in the line instead
        return {name: {"error": f"{type(e).__name__}: {e}"}}


def poisson_stream(collo, workloads, device, budget):
    """Requests of the serving-stream shape at their stated sizes (n log-uniform
    on [5, 100], N on [200, 5000]) arriving at 200 per second, served for a
    bounded time."""
    import numpy as np
    stream = workloads.serving_stream(count=16, rate_hz=200.0)
    probs = [collo.Problem(i, device=device) for _, i in stream]
    srv = collo.Server(16, budget_bytes=budget, device=device, precision=collo.MIXED, tol=TOL)
    srv.set_admission(1)
    limit = 60.0
    t0 = time.perf_counter()
    nxt, tk, done_at = 0, {}, {}
    c0 = srv.counters()
    while len(done_at) < len(stream) and time.perf_counter() - t0 < limit:
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
    c1 = srv.counters()
    res = {j: srv.poll(tk[j]) for j in done_at}
    srv.close()
    for p in probs:
        p.close()
    lat = [1e3 * (done_at[j] - stream[j][0]) for j in done_at]
    return {"poisson_stream": {
        "requests": len(stream), "finished": len(done_at), "wall_s": dt, "limit_s": limit,
        "sizes_n_N": [[i.n, i.N] for _, i in stream],
        "newton_steps_per_s": (c1[0] - c0[0]) / dt,
        "latency_ms": {"p50": float(np.percentile(lat, 50)) if lat else None,
                       "p99": float(np.percentile(lat, 99)) if lat else None},
        "status_counts": {str(s_): sum(1 for r in res.values() if r["status"] == s_)
                          for s_ in sorted(set(r["status"] for r in res.values()))},
        "what": "serving-stream shape at its stated sizes: 16 requests, seeded exponential "
                "gaps at 200/s, each submitted at its arrival time, served for at most "
                f"{limit:.0f} s; latency = arrival to result (host clock)"}}


def cpu_sample(insts):
    """The oracle's bounded sample: the median instance of the batch by
    factorization work."""
    order = sorted(range(len(insts)), key=lambda i: insts[i].N * (8 * insts[i].n + insts[i].p) ** 3)
    return insts[order[len(order) // 2]]


def cpu_baseline(insts):
    from oracle import ipm as oipm
    inst = cpu_sample(insts)
    t0 = time.perf_counter()
    r = oipm.solve(inst, opt=oipm.Options(max_iter=2))
    dt = time.perf_counter() - t0
    from oracle import lifted as olifted
    from oracle.nlp import Problem as OProblem
    from paper_2607_12201_gb300 import workloads
    c2 = workloads.config2()
    op = OProblem(c2)
    lopt = olifted.Options(relax=LIFTED_R)
    st, _ = olifted.initial_point(op, c2.theta0, lopt)
    t1 = time.perf_counter()
    ev = op.evaluate(st.x, st.lam)
    olifted.newton_direction(op, ev, st, lopt.mu_init, 0.0, lopt)
    lifted_s = time.perf_counter() - t1
    return {"value": r.iterations / dt, "unit": "Newton steps/s", "cores": 1,
            "kind": "oracle",
            "lifted_step_config2_N400_s": lifted_s,
            "sample": f"oracle IPM on one instance of the batch (n = {inst.n}, N = {inst.N}, "
                      f"the median by factorization work): initial point + "
                      f"{r.iterations} Newton iterations ({dt:.1f} s, numpy/scipy FP64, one BLAS "
                      "thread, block KKT mode)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1:
        init_dist(world, "gloo")
        if rank != 0:
            return
    from oracle import ipm as oipm
    from paper_2607_12201_gb300 import workloads
    inst = cpu_sample(workloads.multistart_batch())
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
           "config": {"workload": WORKLOAD.format(S=args.slots, B=args.budget_gib),
                      "step": f"oracle initial point + {per} Newton iterations of one instance "
                              f"(n = {inst.n}, N = {inst.N})"},
           "cpu_baseline": {"value": v, "unit": "Newton steps/s", "cores": 1, "kind": "oracle",
                            "sample": f"{args.steps} x (initial point + {per} Newton iterations)"},
           "e2e": {"value": v, "unit": "Newton steps/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def only_phase(args):
    from paper_2607_12201_gb300 import build as B
    B.build()
    from paper_2607_12201_gb300 import collo, workloads
    if args.phase_case == "large":
        one = workloads.random_network(45, 90, log10k=(-2.0, 1.0), n_obs=4, M=50, T=20.0, N=150,
                                       seed=4501, theta0_spread=1.0)
        insts = [one] * args.slots
    else:
        insts = workloads.multistart_batch()[:args.slots]
    probs = [collo.Problem(i) for i in insts]
    for p, i in zip(probs, insts):
        x, _ = p.initial_states(i.theta0)
        p.eval_raw(x.ctypes.data, None)
    ms = collo.batch_time_phase(probs, args.only_phase, collo.MIXED, reps=1)
    print(json.dumps({"only_phase": args.only_phase, "case": args.phase_case,
                      "instances": len(insts), "elements": sum(i.N for i in insts), "ms": ms}),
          flush=True)
    for p in probs:
        p.close()


def only_serve(args):
    from paper_2607_12201_gb300 import build as B
    B.build()
    from paper_2607_12201_gb300 import collo, workloads
    insts = workloads.multistart_batch()
    probs = [collo.Problem(i) for i in insts]
    srv = collo.Server(args.slots, budget_bytes=int(args.budget_gib * (1 << 30)),
                       precision=collo.MIXED, tol=TOL)
    srv.set_admission(args.admit)
    st = Stream(collo, srv, insts, probs, 0)
    l0 = collo.launch_count()
    t0 = time.perf_counter()
    st.step(args.only_serve)
    print(json.dumps({"only_serve": args.only_serve, "wall_s": time.perf_counter() - t0,
                      "counters": srv.counters(), "launches": collo.launch_count() - l0}),
          flush=True)
    srv.close()
    for p in probs:
        p.close()


def phase_profile(args):
    """Per-phase host wall time of the IPM driver over --slice server steps of the
    stream after --warmup slices (COLLO_PROFILE=1: the driver synchronises at
    each phase boundary)."""
    os.environ["COLLO_PROFILE"] = "1"
    from paper_2607_12201_gb300 import build as B
    B.build()
    from paper_2607_12201_gb300 import collo, workloads
    insts = workloads.multistart_batch()
    probs = [collo.Problem(i) for i in insts]
    srv = collo.Server(args.slots, budget_bytes=int(args.budget_gib * (1 << 30)),
                       precision=collo.MIXED, tol=TOL)
    srv.set_admission(args.admit)
    st = Stream(collo, srv, insts, probs, 0)
    for _ in range(args.warmup):
        st.step(args.slice)
    collo.phase_profile(reset=True)
    c0 = srv.counters()
    t0 = time.perf_counter()
    st.step(args.slice)
    wall = time.perf_counter() - t0
    prof = collo.phase_profile(reset=True)
    c1 = srv.counters()
    print(json.dumps({"phase_profile": {k: {"ms": round(v[0], 1), "rounds": v[1]}
                                        for k, v in prof.items()},
                      "wall_s": round(wall, 3), "server_steps": args.slice,
                      "newton_steps": c1[0] - c0[0], "slots": args.slots,
                      "admit_group": args.admit, "tol": TOL}), flush=True)
    srv.close()
    for p in probs:
        p.close()


def main():
    args = parse_args()
    if args.only_next:
        from paper_2607_12201_gb300 import build as B
        B.build()
        from paper_2607_12201_gb300 import collo, workloads
        print(json.dumps(conditions_and_refinement(collo, workloads, 0)), flush=True)
    elif args.only_lifted:
        from paper_2607_12201_gb300 import build as B
        B.build()
        from paper_2607_12201_gb300 import collo, workloads
        print(json.dumps(lifted_comparison(collo, workloads, 0, args.lifted_case)), flush=True)
    elif args.only_phase:
        only_phase(args)
    elif args.only_serve:
        only_serve(args)
    elif args.phase_profile:
        phase_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
