#!/usr/bin/env python
"""Benchmark of the GPU Radau-collocation interior-point path.

Workload: the 10-species / 20-reaction random mass-action network on
N = 400 Radau elements (K = 3), 4 observed species x 50 times, T = 20,
seed 3 (``workloads.config2()``): 16 020 primal unknowns, 16 000
constraints, 20 log10 rate constants.

A timed step is one full interior-point solve (from theta0 to convergence) in
the mixed-precision path (FP32 element factorization and block cyclic
reduction, FP64 parameter Schur complement, residuals and refinement).
``value`` = Newton steps per second over the K timed solves; the plain FP64
path, solves/s, p50/p99 solve latency, an end-to-end number through host
buffers, the dominant kernel's roofline and the CPU oracle are reported
beside it.  Between timed solves the L2 cache is flushed by writing a 256 MiB
buffer (the working set is ~40 MB, smaller than L2).

``--impl reference`` times the CPU oracle instead (a bounded sample: each
step is the oracle's initial point plus two Newton iterations).

Multi-GPU (torchrun, one process per GPU): each rank solves its own copy of
the workload with no collective on the data path (weak scaling); the timed
region is bracketed by barriers and the slowest rank's time is used.
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

WORKLOAD = "massaction_n10_r20_N400_K3 (config 2: 10 species, 20 reactions, N=400, T=20, seed 3)"
METRIC = "Newton steps/s (mixed-precision IPM path, config 2)"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--only-solve", choices=["mixed", "fp64"], default=None,
                    help="run one solve of the workload and exit (for profiler launch lists)")
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


def elem_factor_work(n: int, p: int, N: int, bytes_per: int):
    """Algorithmic flops and bytes of one element-condensation launch.

    Per element: eliminating the 3n interior (state, multiplier) pairs of the
    symmetric (8n + p) block; pair q updates the t(t+1)/2 trailing entries
    (t = 8n + p - 2q - 2) with two FMAs each and forms 2t multipliers with four
    FMAs per row.  Bytes: FP64 derivative blocks read (jac_z, hess_zz at
    3 n^2, jac_theta, hess_ztheta at 3 n p, objective block 16 n doubles) and
    the factor written (6n L columns of length 8n + p, 3n pivots, the 2n x 2n
    interface block, its 2n x p border, the p x p FP64 Schur part)."""
    ext = 8 * n + p
    fl = 0
    for q in range(3 * n):
        t = ext - 2 * q - 2
        fl += 2 * t * (t + 1) + 8 * t
    rd = 8 * (2 * 3 * n * n + 2 * 3 * n * p + 16 * n)
    wr = bytes_per * (6 * n * ext + 9 * n + 4 * n * n + n * n + 2 * n * p) + 8 * p * p
    return fl * N, (rd + wr) * N


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
    dist = init_dist(world, "nccl")
    inst = workloads.config2()
    prob = collo.Problem(inst, device=local)
    stream = torch.cuda.ExternalStream(prob.stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def flush_l2(i):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()

    def timed_solve(prec):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = prob.ipm_solve(precision=prec, want_x=False)
        e1.record(stream)
        e1.synchronize()
        return r, e0.elapsed_time(e1)

    for i in range(args.warmup):
        flush_l2(i)
        timed_solve(collo.MIXED)
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = collo.launch_count()
    its, ms_list, statuses, theta_mixed = [], [], [], None
    for i in range(args.steps):
        flush_l2(i)
        r, ms = timed_solve(collo.MIXED)
        its.append(r["iterations"])
        ms_list.append(ms)
        statuses.append(r["status"])
        theta_mixed = r["theta"]
    launches = collo.launch_count() - l0
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    t_total = reduce_max(sum(ms_list), world)
    its_total = reduce_sum(float(sum(its)), world)
    solves_total = reduce_sum(float(args.steps), world)
    value = its_total / (t_total * 1e-3)

    # plain FP64 path on the same GPU
    k64 = max(1, min(args.steps, 5))
    flush_l2(1)
    timed_solve(collo.FP64)
    ms64, its64, theta64 = [], [], None
    for i in range(k64):
        flush_l2(i)
        r, ms = timed_solve(collo.FP64)
        ms64.append(ms)
        its64.append(r["iterations"])
        theta64 = r["theta"]
    fp64_value = sum(its64) / (sum(ms64) * 1e-3)
    perr = float(np.max(np.abs(theta_mixed - theta64) / np.maximum(np.abs(theta64), 1e-12)))

    # phase timings and the dominant kernel's roofline (CUDA events on the
    # library's stream, after a final mixed solve so its state is current)
    timed_solve(collo.MIXED)
    phases = {}
    for name, ph, prec in [("eval", 3, -1), ("factor_fp32", 1, collo.MIXED),
                           ("solve_fp32", 2, collo.MIXED), ("forward_sweep", 4, -1),
                           ("elem_condense_fp32", 0, collo.MIXED)]:
        phases[name] = prob.time_phase(ph, prec, reps=20)
    timed_solve(collo.FP64)
    for name, ph, prec in [("factor_fp64", 1, collo.FP64), ("solve_fp64", 2, collo.FP64),
                           ("elem_condense_fp64", 0, collo.FP64)]:
        phases[name] = prob.time_phase(ph, prec, reps=20)
    fl32, by32 = elem_factor_work(inst.n, inst.p, inst.N, 4)
    peak32 = collo.alu_peak(collo.MIXED)
    peak64 = collo.alu_peak(collo.FP64)
    hbm = measured_peaks().get("hbm_gbs")
    t_el = phases["elem_condense_fp32"] * 1e-3
    ach_fl = fl32 / t_el / 1e12
    ach_by = by32 / t_el / 1e9
    # the roof that bounds this kernel: compare its compute and memory times at the peaks
    if hbm and by32 / (hbm * 1e9) > fl32 / (peak32 * 1e12):
        roof = {"bound": "hbm", "achieved": ach_by, "peak": hbm, "unit": "GB/s",
                "frac": ach_by / hbm, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    else:
        roof = {"bound": "alu", "achieved": ach_fl, "peak": peak32, "unit": "TFLOP/s",
                "frac": ach_fl / peak32,
                "peak_source": "measured live: FP32 FFMA throughput probe (collo_alu_peak)"}
    roof.update({"kernel": "k_elem_factor<float> (element condensation)",
                 "algorithmic_flops": fl32, "algorithmic_bytes": by32, "ms": phases["elem_condense_fp32"],
                 "traffic": None})
    fl64, _ = elem_factor_work(inst.n, inst.p, inst.N, 8)
    fp64_kernel = {"kernel": "k_elem_factor<double>", "ms": phases["elem_condense_fp64"],
                   "achieved_tflops": fl64 / (phases["elem_condense_fp64"] * 1e-3) / 1e12,
                   "fp64_peak_tflops": peak64}

    out = {
        "metric": METRIC, "value": value, "unit": "Newton steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp32 factor + fp64 residual/refinement",
        "data": "synthetic (seeded mass-action network, noisy observations)",
        "config": {"workload": WORKLOAD, "step": "one full IPM solve from theta0",
                   "newton_steps_per_solve": statistics.mean(its),
                   "n_x": prob.n_x, "n_c": prob.n_c, "p": inst.p,
                   "l2": "flushed between timed solves (256 MiB write)",
                   "parallelism": f"replicas x{world}"},
        "solves_per_s": solves_total / (t_total * 1e-3),
        "latency_ms": {"p50": float(np.percentile(ms_list, 50)),
                       "p99": float(np.percentile(ms_list, 99))},
        "status": sorted(set(statuses)),
        "fp64_path": {"newton_steps_per_s": fp64_value,
                      "solves_per_s": k64 / (sum(ms64) * 1e-3),
                      "ms_per_solve": sum(ms64) / k64, "solves": k64},
        "mixed_vs_fp64_speedup": value / fp64_value,
        "param_rel_err_vs_fp64": perr,
        "phases_ms": phases, "roofline": roof, "fp64_elem_kernel": fp64_kernel,
        "gpu_launches": launches, "clocks": clk,
    }
    if not args.no_e2e:
        k_e = max(1, min(args.steps, 5))
        keep = [inst.react, inst.prod, inst.pidx, inst.kfix, inst.x0, inst.theta_lo,
                inst.theta_hi, inst.obs_t, inst.obs_s, inst.obs_y, inst.obs_sigma, inst.theta0]
        h2d = int(sum(np.asarray(a).nbytes for a in keep))
        tot, its_e = 0.0, 0
        for i in range(k_e):
            flush_l2(i)
            t0 = time.perf_counter()
            with collo.Problem(inst, device=local) as p2:
                r = p2.ipm_solve(precision=collo.MIXED, want_x=False)
            t1 = time.perf_counter()
            tot += t1 - t0
            its_e += r["iterations"]
        tot = reduce_max(tot, world)
        its_e = reduce_sum(float(its_e), world)
        out["e2e"] = {"value": its_e / tot, "unit": "Newton steps/s",
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8 * inst.p + 8,
                      "what": "collo_problem_create from host arrays + collo_ipm_solve + "
                              "theta* read back, per solve", "solves": k_e}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(inst, iters=6)
    if rank == 0:
        print(json.dumps(out), flush=True)
    prob.close()


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
           "config": {"workload": WORKLOAD,
                      "step": f"oracle initial point + {per} Newton iterations"},
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


def main():
    args = parse_args()
    if args.only_solve:
        only_solve(args.only_solve)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
