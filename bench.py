#!/usr/bin/env python
"""Benchmark of the GPU Radau-collocation interior-point path.

Workload: the 10-species / 20-reaction random mass-action network on
N = 400 Radau elements (K = 3), 4 observed species x 50 times, T = 20,
seed 3 (``workloads.config2()``): 16 020 primal unknowns, 16 000 constraints,
20 log10 rate constants, solved from B seeded starting points
theta_true + U[-0.1, 0.1] (a multistart run, ``--batch``, default 64).

A timed step is one batched solve: all B starts advance together, one Newton
step per iteration of the lock-step driver, every phase one launch over all
unfinished instances, in the mixed-precision path (FP32 element
factorization and block cyclic reduction, FP64 parameter Schur complement,
residuals and refinement, FP64 factorization once mu < 1e-6).  ``value`` =
Newton steps per second summed over the batch.  Beside it: the same path and
the plain FP64 path on a single instance, per-instance latency percentiles,
an end-to-end number through host buffers, the dominant kernel's roofline,
the CPU oracle.  Between timed steps the L2 cache is flushed (256 MiB write).

``--impl reference`` times the CPU oracle instead (a bounded sample: each step
is the oracle's initial point plus two Newton iterations of one instance).

Multi-GPU (torchrun, one process per GPU): each rank solves its own batch
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

WORKLOAD = ("massaction_n10_r20_N400_K3 x {B} multistart (config 2: 10 species, 20 reactions, "
            "N=400, T=20, seed 3; starts theta_true + U[-0.1,0.1])")
METRIC = "Newton steps/s (mixed-precision batched IPM path, config 2 multistart)"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--only-solve", choices=["mixed", "fp64"], default=None,
                    help="run one single-instance solve and exit (for profiler launch lists)")
    ap.add_argument("--only-batch", action="store_true",
                    help="run one batched solve and exit (for profiler launch lists)")
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
    nb = args.batch
    starts = workloads.multistart_thetas(inst, nb, seed=2002 + rank)
    probs = [collo.Problem(inst, device=local) for _ in range(nb)]
    stream = torch.cuda.ExternalStream(probs[0].stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def flush_l2(i):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()

    def timed_batch(prec):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = collo.batch_solve(probs, theta0s=starts, precision=prec)
        e1.record(stream)
        e1.synchronize()
        return res, e0.elapsed_time(e1)

    for i in range(args.warmup):
        flush_l2(i)
        timed_batch(collo.MIXED)
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = collo.launch_count()
    its, ms_list, statuses, lat, last = 0, [], [], [], None
    for i in range(args.steps):
        flush_l2(i)
        res, ms = timed_batch(collo.MIXED)
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
    solves_total = reduce_sum(float(args.steps * nb), world)
    value = its_total / (t_total * 1e-3)

    # single-instance paths on the same GPU: mixed and the plain FP64 path
    one = probs[0]
    single = {}
    for name, prec in [("mixed", collo.MIXED), ("fp64", collo.FP64)]:
        one.ipm_solve(theta0=starts[0], precision=prec, want_x=False)
        ms_s, its_s, th = [], 0, None
        for i in range(3):
            flush_l2(i)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = one.ipm_solve(theta0=starts[0], precision=prec, want_x=False)
            e1.record(stream)
            e1.synchronize()
            ms_s.append(e0.elapsed_time(e1))
            its_s += r["iterations"]
            th = r["theta"]
        single[name] = {"newton_steps_per_s": its_s / (sum(ms_s) * 1e-3),
                        "solves_per_s": len(ms_s) / (sum(ms_s) * 1e-3),
                        "ms_per_solve": sum(ms_s) / len(ms_s), "theta": th}
    # parameter error of the batched mixed path against single-instance FP64 solves
    perr = 0.0
    for j in range(min(4, nb)):
        r64 = one.ipm_solve(theta0=starts[j], precision=collo.FP64, want_x=False)
        if r64["status"] in (collo.OK, collo.ACCEPTABLE):
            th = last[j]["theta"]
            perr = max(perr, float(np.max(np.abs(th - r64["theta"]) /
                                          np.maximum(np.abs(r64["theta"]), 1e-12))))

    # dominant kernel (batched factorization) and phase timings with CUDA events
    timed_batch(collo.MIXED)
    ph = {"factor_fp32": collo.batch_time_phase(probs, 1, collo.MIXED, reps=5),
          "solve_fp32": collo.batch_time_phase(probs, 2, collo.MIXED, reps=5),
          "eval": collo.batch_time_phase(probs, 3, collo.MIXED, reps=5)}
    fl32, by32 = factor_work(inst.n, inst.p, inst.N, 4)
    fl32 *= nb
    by32 *= nb
    peak32 = collo.alu_peak(collo.MIXED)
    peak64 = collo.alu_peak(collo.FP64)
    hbm = measured_peaks().get("hbm_gbs")
    t_f = ph["factor_fp32"] * 1e-3
    ach_fl, ach_by = fl32 / t_f / 1e12, by32 / t_f / 1e9
    if hbm and by32 / (hbm * 1e9) > fl32 / (peak32 * 1e12):
        roof = {"bound": "hbm", "achieved": ach_by, "peak": hbm, "unit": "GB/s",
                "frac": ach_by / hbm, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    else:
        roof = {"bound": "alu", "achieved": ach_fl, "peak": peak32, "unit": "TFLOP/s",
                "frac": ach_fl / peak32,
                "peak_source": "measured live: FP32 FFMA throughput probe (collo_alu_peak)"}
    roof.update({"kernel": f"k_factor_b<float> (batched factorization, {nb} instances)",
                 "algorithmic_flops": fl32, "algorithmic_bytes": by32,
                 "ms": ph["factor_fp32"], "traffic": None,
                 "other_roof": {"alu_tflops": ach_fl, "alu_peak_tflops": peak32,
                                "hbm_gbs": ach_by, "hbm_peak_gbs": hbm}})

    out = {
        "metric": METRIC, "value": value, "unit": "Newton steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp32 factor + fp64 residual/refinement",
        "data": "synthetic (seeded mass-action network, noisy observations, seeded starts)",
        "config": {"workload": WORKLOAD.format(B=nb), "batch": nb,
                   "step": f"one batched solve of {nb} starts from theta0 to convergence",
                   "newton_steps_per_step": its / max(args.steps, 1),
                   "n_x_per_instance": one.n_x, "n_c_per_instance": one.n_c, "p": inst.p,
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{world} (independent batches)"},
        "solves_per_s": solves_total / (t_total * 1e-3),
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "what": "per-instance time from batch start to that instance's result"},
        "status_counts": {str(s): statuses.count(s) for s in sorted(set(statuses))},
        "single_instance": {k: {kk: vv for kk, vv in v.items() if kk != "theta"}
                            for k, v in single.items()},
        "speedup_vs_fp64_single": value / single["fp64"]["newton_steps_per_s"],
        "param_rel_err_vs_fp64": perr,
        "phases_ms": ph, "roofline": roof,
        "peaks_tflops": {"fp32_ffma": peak32, "fp64_dfma": peak64},
        "gpu_launches": launches, "clocks": clk,
    }
    if not args.no_e2e:
        keep = [inst.react, inst.prod, inst.pidx, inst.kfix, inst.x0, inst.theta_lo,
                inst.theta_hi, inst.obs_t, inst.obs_s, inst.obs_y, inst.obs_sigma]
        h2d = nb * int(sum(np.asarray(a).nbytes for a in keep)) + 8 * inst.p * nb
        tot, its_e = 0.0, 0
        k_e = max(1, min(args.steps, 3))
        for i in range(k_e):
            flush_l2(i)
            t0 = time.perf_counter()
            ps = [collo.Problem(inst, device=local) for _ in range(nb)]
            res = collo.batch_solve(ps, theta0s=starts, precision=collo.MIXED)
            for pb in ps:
                pb.close()
            t1 = time.perf_counter()
            tot += t1 - t0
            its_e += sum(r["iterations"] for r in res)
        tot = reduce_max(tot, world)
        its_e = reduce_sum(float(its_e), world)
        out["e2e"] = {"value": its_e / tot, "unit": "Newton steps/s",
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": nb * (8 * inst.p + 64),
                      "what": f"{nb} x collo_problem_create from host arrays + "
                              "collo_batch_solve + theta* read back, per step", "steps": k_e}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(inst, iters=6)
    if rank == 0:
        print(json.dumps(out), flush=True)
    for pb in probs:
        pb.close()


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
           "config": {"workload": WORKLOAD.format(B=args.batch),
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
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
