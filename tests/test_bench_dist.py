"""Multi-process path of bench.py on CPU (gloo, world size 2): the timing
reductions take the maximum time and the summed work over ranks, and ranks
meet at the barriers that bracket the timed region."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist
    bench.init_dist(world, "gloo")
    bench.barrier(world)
    t = bench.reduce_max(1.0 + rank, world)
    s = bench.reduce_sum(10.0 * (rank + 1), world)
    bench.barrier(world)
    out[rank] = (t, s)
    dist.destroy_process_group()


def test_reductions_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == out[1] == (2.0, 30.0)


def test_single_rank_helpers_are_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.reduce_sum(2.0, 1) == 2.0
    bench.barrier(1)


def test_factor_work_counts():
    import bench
    # one 2x2 pivot of a 4x4 block: t = 2 trailing rows -> 2*2*3 + 8*2 flops
    assert bench._pair_flops(4, 1) == 2 * 2 * 3 + 8 * 2
    # its L columns have 2 rows each below the pair
    assert bench._pair_l_entries(4, 1) == 4
    # one species, no parameter, one element: element block 8 rows (3 pairs:
    # 2 (6 + 4 + 2) = 24 L entries), reduction block 4 rows (1 pair: 4 entries),
    # 12 pivot values, 8 KKT unknowns, 10 intermediate values; FP32 factors:
    # 2*4*(28 + 12) + 8*2*8 + 2*4*10 = 528 bytes
    assert bench.solve_bytes(1, 0, 1, 4) == 528
    fe, be = bench.elem_factor_work(10, 20, 400, 4)
    fr, br = bench.reduction_work(10, 20, 400, 4)
    assert fe > fr > 0 and be > 0 and br > 0


REQUIRED = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
            "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
            "cpu_baseline", "e2e"}


def _json_lines(text):
    import json
    return [json.loads(l) for l in text.splitlines() if l.startswith("{")]


def _check_reference_line(line, n):
    assert REQUIRED <= set(line)
    assert line["impl"] == "reference" and line["n_gpus"] == n
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 0
    assert "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_prints_one_contract_line():
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_reference_line(lines[0], 1)


def test_reference_arm_under_torchrun_prints_once_from_rank_0():
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_reference_line(lines[0], 2)


def test_clock_sampler_summarises_nvidia_smi_samples(tmp_path):
    # the median SM clock under load, the maximum clock, and every throttle reason
    # seen active; malformed and N/A lines are skipped
    import bench

    class _Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    csv = tmp_path / "clocks.csv"
    csv.write_text(
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
        "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active\n"
        "0, 2010, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
        "0, [N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
        "garbage line\n")
    s = bench.ClockSampler(0)
    s.proc, s.path = _Done(), str(csv)
    out = s.stop()
    assert out["sm_mhz"] == 2010.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    assert not csv.exists()
    s2 = bench.ClockSampler(0)
    assert s2.stop()["reasons"] == ["nvidia-smi unavailable"]
