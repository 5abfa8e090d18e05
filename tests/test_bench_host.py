"""Host-side logic of bench.py, on CPU: the replica aggregation at world
size 2 (gloo ranks launched by torch.distributed.run), the clock-sample
summary, and the rank rule of the reference arm."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

RANK_SCRIPT = r'''
import json, os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
ms = [10.0, 25.0][rank]            # the second replica is the slow one
ms_max = bench.reduce_max(ms, world, device="cpu")
rate = bench.replica_throughput(3.0e9, ms_max, world)
with open(os.path.join({out!r}, f"rank{{rank}}.json"), "w") as f:
    json.dump({{"rank": rank, "world": world, "ms_max": ms_max, "rate": rate}}, f)
dist.destroy_process_group()
'''


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_replica_max_over_two_gloo_ranks(tmp_path):
    script = tmp_path / "rank.py"
    script.write_text(RANK_SCRIPT.format(root=ROOT, out=str(tmp_path)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), str(script)]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=240)
    assert r.returncode == 0, r.stderr[-2000:]
    outs = [json.loads((tmp_path / f"rank{k}.json").read_text()) for k in range(2)]
    for o in outs:
        assert o["world"] == 2
        assert o["ms_max"] == 25.0                      # the slowest replica's time
        assert abs(o["rate"] - 2 * 3.0e9 / 25e-3) < 1e-3  # units of both ranks / that time


def test_replica_helpers_at_world_one():
    assert bench.reduce_max(7.5, 1) == 7.5
    assert bench.replica_throughput(12.0e9, 2.0, 1) == pytest.approx(6.0e12)


def smi(sm, reason_cols):
    return f"0, {sm}, 2070, 900.0, " + ", ".join(reason_cols)


NA = ["Not Active"] * 4


def test_clock_summary_window_and_reasons():
    samples = [(0.0, smi(1200, NA)),                                  # before the region
               (1.0, smi(2070, NA)),
               (1.2, smi(2040, NA[:3] + ["Active"])),                 # power cap: kept, noted
               (1.4, smi(2010, NA)),
               (9.0, smi(900, ["Active"] + NA[1:]))]                  # after the region
    s = bench.summarize_clocks(samples, 0.9, 1.5)
    assert s == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    # a region shorter than the sampling period takes the nearest samples
    s = bench.summarize_clocks(samples, 1.05, 1.1)
    assert s["samples"] == 2 and s["sm_mhz"] == pytest.approx(0.5 * (2070 + 2040))
    # header or malformed lines are skipped; nothing parsed gives None
    assert bench.summarize_clocks([(0.0, "index, clocks.sm [MHz]"), (0.1, "garbage")]) is None
    s = bench.summarize_clocks([(0.0, smi(2070, ["Active", "Active", "Not Active", "Not Active"]))])
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       capture_output=True, text=True, timeout=120, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line_on_small_workload():
    """The reference arm times the oracle on the host and prints the contract
    line with impl = reference and its own e2e (no transfers)."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "heat2d-20", "--steps", "2", "--warmup", "1", "--cpu-iters", "8"],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_fp64_roofline_counts_the_unit_form():
    """The FP64 roofline's algorithmic work: 7 FP64 instructions a grid point
    (3 pair sums, 4 FMAs; w stored divided by s_j kappa_x), 6 in the first
    iteration, averaged over the m launches of a query."""
    import workloads as W
    p = W.heat((40, 30, 20), block=(4, 4, 4), output="centre", dt=0.1, steps=5, m=30)
    n = 40 * 30 * 20
    assert bench.fp64_instr_per_launch(p) == pytest.approx(n * (6 + 7 * 29) / 30)
