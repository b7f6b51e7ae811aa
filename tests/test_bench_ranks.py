"""The multi-rank form of bench.py (one independent replica per rank): the
whole-job value takes the slowest rank's time and the sum of the ranks' work.
Run as two gloo ranks on the CPU; no GPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
rank, world, _ = bench.dist_env()
dist.init_process_group("gloo", init_method="env://")
ms, flips, e2e = bench.reduce_over_ranks(dist, "cpu", 100.0 + 50.0 * rank, 1000 * (rank + 1), 7.0 + rank)
print(json.dumps({"rank": rank, "world": world, "ms": ms, "flips": flips, "e2e": e2e}), flush=True)
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reduce_max_time_and_summed_work():
    pytest.importorskip("torch")
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["world"] == 2
        assert o["ms"] == 150.0  # the slowest rank
        assert o["flips"] == 3000.0  # 1000 + 2000
        assert o["e2e"] == 15.0


def test_single_rank_passes_through():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks(None, "cpu", 12.5, 40, 3.0) == (12.5, 40.0, 3.0)


def test_reference_arm_runs_on_rank_zero_only():
    """--impl reference under torchrun: rank 0 times the oracle, the others exit 0 without work."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_clock_record_keeps_the_timed_region_and_every_throttle_reason():
    sys.path.insert(0, ROOT)
    import datetime

    import bench

    def row(t, sm, reasons=("Not Active",) * 4, uuid="GPU-a"):
        ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return ", ".join([ts, "0", uuid, str(sm), "2070", "900.0", "0x0"] + list(reasons))

    t0 = 1_800_000_000.0
    lines = [row(t0 - 0.5, 1000),  # before the region: idle clock, left out
             row(t0 + 0.1, 2070), row(t0 + 0.3, 2070),
             row(t0 + 0.5, 1800, ("Not Active", "Not Active", "Not Active", "Active")),
             row(t0 + 0.6, 2000, uuid="GPU-b"),  # another GPU
             row(t0 + 2.0, 500)]  # after the region
    rec = bench.summarize_clocks(lines, "GPU-a", t0, t0 + 1.0)
    assert rec["samples"] == 3
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]
    hot = bench.summarize_clocks([row(t0, 1500, ("Active", "Not Active", "Not Active", "Not Active"))], None)
    assert hot["reasons"] == ["hw_slowdown"]
    assert bench.summarize_clocks([], None)["reasons"] == ["no samples"]


def test_converge_report_compares_with_the_oracle_values():
    """bench.py --converge compares a converged run with the oracle's stored
    run of the same seed and with the oracle's seed mean, bin by bin."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench

    with open(os.path.join(root, "tests", "golden", "potts10_L8_converged.json")) as f:
        ref = json.load(f)
    r1 = ref["runs"][0]
    same = {k: r1[k] for k in ("c_peak_T", "c_peak", "Tc_equal_peak", "E_peaks")}
    lng = [m if m is not None else float("-inf") for m in ref["lng_mean"]]
    out = bench.oracle_reference("potts10_L8", r1["seed"], same, lng)
    assert out["same_as_oracle"] is True
    assert out["oracle_seeds"] == len(ref["runs"])
    assert out["lng_within_3sd"] == 1.0 and out["lng_max_abs_z"] == 0.0
    assert out["lng_bins"] == sum(m is not None for m in ref["lng_mean"])
    moved = dict(same, c_peak_T=same["c_peak_T"] * 1.001)
    assert bench.oracle_reference("potts10_L8", r1["seed"], moved, None)["same_as_oracle"] is False
    assert bench.oracle_reference("potts10_L8", 99, same, None).get("oracle_same_seed") is None
    assert bench.oracle_reference("no_such_workload", 1, same, None) is None


def test_pipe_bounds_take_the_smallest_pipe():
    """The per-flip roofline: each pipe's rate x SMs x clock / its operations
    per flip; with GB300's measured rates the FP64 pipe binds once exp is
    charged for the decisions with D < 0, and the issue bound equals
    152 x 128 lanes x f / 103."""
    import bench

    pipes = {"sms": 152, "dadd": 1.68, "imad": 64.2, "imad_hi": 32.0, "lop3": 64.2, "iadd": 128.6, "lds": 23.0}
    f = 2.07e9
    b = bench.pipe_bounds(pipes, f, 0.62)
    assert min(b, key=b.get) == "fp64"
    assert abs(b["issue"] - 152 * 128 * f / 103) < 1e-3 * b["issue"]
    assert abs(b["fp64"] - 152 * 1.68 * f / (2 + 20 * 0.62)) < 1e-6 * b["fp64"]
    assert bench.pipe_bounds(pipes, f, 0.0)["fp64"] > b["fp64"]  # no exp charged: a higher bound


def test_bench_modes_parse():
    import sys

    import bench

    argv = sys.argv
    try:
        sys.argv = ["bench.py", "--weak-scaling", "potts10_L20,potts10_L40_w291", "--converge-limit", "60"]
        a = bench.parse_args()
        assert a.weak_scaling.split(",") == ["potts10_L20", "potts10_L40_w291"] and a.converge_limit == 60
        sys.argv = ["bench.py", "--production", "--autotune", "--instances", "512", "--converge-save", "d"]
        a = bench.parse_args()
        assert a.production and a.autotune and a.instances == 512 and a.converge_save == "d"
    finally:
        sys.argv = argv
