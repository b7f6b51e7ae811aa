#!/usr/bin/env python3
"""Benchmark of the REWL hot path (arXiv:1312.3004, Sec. 2) on one GB300.

Workload (default): 10-state Potts model, L = 80 (N = 6400) on a torus,
h = 64 windows with 75% overlap, m = 16 walkers per window (1024 walkers),
4-bit packed spins, FP64 ln g, 10^4 WL steps per walker between exchanges,
ln f_final = 1e-8, flatness 0.8; synthetic (seeded) initial states.

One step = one exchange round: K WL proposals for every walker of every
unfinished window (sweep kernel), then flatness / merge / f-reduction (check
kernel) and the replica exchange (exchange kernel).  Reported value: WL flip
attempts per second over the timed steps (device events on the launching
stream), L2 flushed between steps.  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (torchrun) every rank runs an independent replica (seed + rank):
there is no data exchange between instances, so scaling is weak.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Algorithmic operations of one WL proposal (what the method needs per flip,
# not what a kernel issues), by the pipe that executes them:
#   Philox4x32-10: 10 rounds x (2 wide multiplies [imad] + 2 three-input
#     XORs [alu]) + 2 counter words [alu]
#   site = r0 N >> 32, new value, y = s / L (high multiplies) and x = s - yL
#     [imad 4]; four wrapped neighbour indices [alu 10]
#   5 spin reads [lsu 5] and their 4-bit extraction [alu 10]
#   dE: 8 compares + 7 adds [alu 15]
#   window test 2, accept compare 1, u construction 4 [alu 7]; two ln g
#     reads [lsu 2]
#   conditional spin write [alu 2, lsu 1]; ln g store [lsu 1]; H read, add,
#     store [lsu 2, alu 1]
#   binary64: D = ln g(E) - ln g(E') and ln g(E) += ln f (2 adds), and exp(D)
#     when D < 0, about 20 binary64 operations (a fraction rho_neg of the
#     decisions, measured on the same workload by the oracle)
OPS_PER_FLIP = {"imad": 24, "alu": 68, "lsu": 11}
ALG_OPS_PER_FLIP = sum(OPS_PER_FLIP.values())  # 103 issue slots of integer / logic / shared-memory work
FP64_PER_FLIP, FP64_PER_EXP = 2, 20
SMS = 152
LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
# DRAM bytes (read + write) of one sweep launch, from ncu captures of the
# current kernels (profiles/sweep_fast_potts10_L80.md, profiles/batch_walker_batched2048.md)
TRAFFIC_PER_LAUNCH = {"potts10_L80": 10.12e6, "batched2048": 6.16e9}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=800)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="potts10_L80",
                    help="potts10_L80 (default), potts10_L300 (the paper's size), potts10_L20, ising_L8, "
                         "batched2048, serving (small jobs) or serving_full (the stated sizes, cost-capped)")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--schedule", default="halving", choices=["halving", "inv_t"],
                    help="inv_t: every window starts in the 1/t stage (ln f = bins / steps, not a power of "
                         "two, so every WL step takes the binary64 add)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--jobs", type=int, default=100, help="arrivals of the serving trace")
    ap.add_argument("--weak-scaling", default="",
                    help="comma-separated workloads run together to convergence (one seed, --converge-limit)")
    ap.add_argument("--production", action="store_true",
                    help="time fixed-weight production rounds (H(E,O)) on the workload after --warmup WL rounds")
    ap.add_argument("--autotune", action="store_true",
                    help="single-instance workloads: time every lane width first (rewl_autotune) and keep the fastest")
    ap.add_argument("--instances", type=int, default=2048,
                    help="batched2048: instances of the batch (fewer only for small profiler captures)")
    ap.add_argument("--cost-cap", type=float, default=1e10,
                    help="serving_full: jobs whose estimated cost exceeds this many proposals are left out")
    ap.add_argument("--converge", default="",
                    help="comma-separated seeds: time each run to ln f < ln f_final instead of timing rounds")
    ap.add_argument("--converge-limit", type=float, default=1800.0, help="seconds per seed before giving up")
    ap.add_argument("--converge-save", default="",
                    help="with --concurrent: save each unfinished seed's state and seconds here at the end")
    ap.add_argument("--converge-resume", default="",
                    help="with --concurrent: continue the seeds saved here (their seconds are added)")
    ap.add_argument("--ref-chunk", type=int, default=32,
                    help="--impl reference: walkers advanced by K WL steps in one timed step")
    ap.add_argument("--concurrent", action="store_true",
                    help="with --converge: run the seeds at the same time, one stream each (for small "
                         "workloads that leave most SMs idle)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_over_ranks(dist, device, total_ms, flips, e2e_flips_per_s):
    """Whole-job figures of independent replicas: the slowest rank's timed
    duration, and the work (and end-to-end rate) summed over the ranks."""
    if dist is None:
        return total_ms, float(flips), e2e_flips_per_s
    import torch

    mx = torch.tensor([total_ms], dtype=torch.float64, device=device)
    sm = torch.tensor([float(flips), e2e_flips_per_s], dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx.item()), float(sm[0].item()), float(sm[1].item())


# ---------------------------------------------------------------------------
def summarize_clocks(lines, uuid=None, t0=None, t1=None):
    """The clock record of a timed region from nvidia-smi CSV rows
    (timestamp, index, uuid, clocks.sm, clocks.max.sm, power, active reasons,
    hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap):
    median SM clock under load, its maximum, and every throttle reason seen.
    Rows outside [t0, t1] (epoch seconds) are left out when the region holds
    any."""
    import datetime

    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 11 or (uuid and parts[2] != uuid):
            continue
        try:
            ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            ts = None
        rows.append((ts, parts[1:]))
    if t0 is not None and t1 is not None:
        inside = [r for r in rows if r[0] is not None and t0 <= r[0] <= t1]
        if inside:
            rows = inside
    rows = [r for _, r in rows]
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(rows)}


class NvmlSampler:
    """SM clock and clock-event reasons read through NVML (the driver's
    libnvidia-ml, by ctypes) every 2 ms from a thread during the timed region:
    a timed region of a few tens of milliseconds still gets a dozen samples.
    Reading only; nothing is set."""

    # nvmlClocksEventReason bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, uuid):
        import ctypes as C
        import threading

        self.C, self.threading = C, threading
        self.lib = C.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = C.c_void_p()
        if not uuid or self.lib.nvmlDeviceGetHandleByUUID(str(uuid).encode(), C.byref(self.h)) != 0:
            raise OSError("no NVML handle for %s" % uuid)
        mx = C.c_uint(0)
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, C.byref(mx))  # 1 = NVML_CLOCK_SM
        self.max_mhz = float(mx.value)
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self.reasons_fn = fn if fn is not None else self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self.samples, self.stop_flag, self.thread = [], False, None

    def _run(self):
        C = self.C
        clk, rs = C.c_uint(0), C.c_ulonglong(0)
        while not self.stop_flag:
            t = time.time()
            if self.lib.nvmlDeviceGetClockInfo(self.h, 1, C.byref(clk)) == 0:
                r = rs.value if self.reasons_fn(self.h, C.byref(rs)) == 0 else 0
                self.samples.append((t, float(clk.value), int(r)))
            time.sleep(0.002)

    def start(self):
        self.thread = self.threading.Thread(target=self._run, daemon=True)
        self.thread.start()

    def stop(self, t0=None, t1=None):
        self.stop_flag = True
        self.thread.join()
        rows = [x for x in self.samples if t0 is None or t1 is None or t0 <= x[0] <= t1] or self.samples
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["no samples"], "source": "nvml"}
        reasons = sorted({name for _, _, r in rows for bit, name in self.REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median(x[1] for x in rows), "sm_min_mhz": min(x[1] for x in rows),
                "sm_max_mhz": self.max_mhz, "reasons": reasons, "samples": len(rows), "source": "nvml, every 2 ms"}


def clock_sampler(uuid):
    """NVML sampling when the driver library answers, else nvidia-smi's."""
    try:
        return NvmlSampler(uuid)
    except Exception:
        return ClockSampler(uuid)


class ClockSampler:
    """nvidia-smi samples every 100 ms around the timed region."""

    FIELDS = ("timestamp,index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self, t0=None, t1=None):
        """Stop sampling; the record of the samples taken in [t0, t1] (epoch s)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        return summarize_clocks(lines, self.uuid, t0, t1)


# ---------------------------------------------------------------------------
def cpu_baseline(p, seed, budget_s):
    """The oracle, as it stands, on this host: rounds of the same workload until
    about budget_s seconds of CPU work (at least one round)."""
    from oracle import oracle as O
    from paper_1312_3004_gb300 import workloads as WL

    t0 = time.perf_counter()
    orc = O.OracleREWL(*WL.rewl_args(p, seed))
    t_create = time.perf_counter() - t0
    rounds, t_run = 0, 0.0
    walkers = p["h"] * p["m"]
    while t_run < budget_s and rounds < 1000:
        t0 = time.perf_counter()
        orc.run(1)
        t_run += time.perf_counter() - t0
        rounds += 1
    flips = rounds * walkers * p["exchange_interval"]
    n_dec, n_neg = orc.decision_counts()
    return {"value": flips / t_run, "unit": "flips/s", "cores": 1, "kind": "oracle",
            "rho_neg": n_neg / max(1, n_dec),
            "sample": "%d exchange round(s) of the %d-walker workload (%d WL proposals, %.1f s), "
                      "after a %.1f s set-up; single-threaded C" % (rounds, walkers, flips, t_run, t_create)}


def run_reference(args):
    """The reference arm: the CPU oracle timed on the host cores.  One step is
    a bounded sample of a round: K WL steps for each of a chunk of walkers, in
    walker order, with the round's barrier (flatness, merge, exchange) after
    the chunk that completes the round, so that --steps K of the default size
    end within seconds."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1312_3004_gb300 import workloads as WL

    p = WL.params(args.workload)
    orc = O.OracleREWL(*WL.rewl_args(p, args.seed))
    walkers = p["h"] * p["m"]
    chunk = max(1, min(walkers, args.ref_chunk))
    K = p["exchange_interval"]
    pos = [0]

    def step():
        g0 = pos[0]
        g1 = min(g0 + chunk, walkers)
        for g in range(g0, g1):
            orc.wl_steps(g, K)
        if g1 == walkers:
            orc.barrier()
            g1 = 0
        pos[0] = g1
        return (g1 - g0 if g1 else walkers - g0) * K

    for _ in range(args.warmup):
        step()
    flips = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        flips += step()
    dt = time.perf_counter() - t0
    value = flips / dt
    line = {
        "impl": "reference", "metric": "flip attempts/s", "value": value, "unit": "flips/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(args.workload, p),
        "cpu_baseline": {"value": value, "unit": "flips/s", "cores": 1, "kind": "oracle",
                         "sample": "each step: %d WL steps for each of %d of the %d walkers (a chunk of an exchange "
                                   "round; the round's barrier runs after its last chunk); %d steps after %d warm-up"
                                   % (K, chunk, walkers, args.steps, args.warmup)},
        "e2e": {"value": value, "unit": "flips/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(name, p):
    return {"workload": name, "q": p["q"], "L": p["L"], "h": p["h"], "overlap": p["overlap"],
            "m": p["m"], "walkers": p["h"] * p["m"], "exchange_interval": p["exchange_interval"],
            "lnf_final": p["lnf_final"], "flatness": p["flatness"], "spin_bits": p["spin_bits"],
            "l2": "flushed between steps (256 MiB write)"}


def pipe_bounds(pipes, f_hz, rho):
    """Flips per second each pipe allows: its measured issue rate x SMs x the SM
    clock / the algorithmic operations per flip it executes."""
    nsm = pipes["sms"]
    return {
        "issue": nsm * LANES_PER_SM * f_hz / ALG_OPS_PER_FLIP,
        "imad": nsm * min(pipes["imad"], pipes["imad_hi"]) * f_hz / OPS_PER_FLIP["imad"],
        "alu": nsm * min(pipes["lop3"], pipes["iadd"]) * f_hz / OPS_PER_FLIP["alu"],
        "lsu": nsm * pipes["lds"] * f_hz / OPS_PER_FLIP["lsu"],
        "fp64": nsm * pipes["dadd"] * f_hz / (FP64_PER_FLIP + FP64_PER_EXP * rho),
    }


# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    from paper_1312_3004_gb300 import REWL, RewlError, _lib
    from paper_1312_3004_gb300 import workloads as WL

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    p = WL.params(args.workload)
    stream = torch.cuda.Stream()
    r = REWL(*WL.rewl_args(p, args.seed + rank), spin_bits=p["spin_bits"], stream=stream)
    if args.schedule == "inv_t":
        r.set_option(_lib.OPT_SCHEDULE, _lib.SCHEDULE_INV_T)
        r.set("phase", 1)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def one_step(ev):
        e0, e1, e2 = ev
        e0.record(stream)
        r.run_phase(_lib.PHASE_SWEEP)
        e1.record(stream)
        r.run_phase(_lib.PHASE_CHECK)
        r.run_phase(_lib.PHASE_EXCHANGE)
        e2.record(stream)

    tuned = r.autotune(2) if args.autotune else None  # ordinary rounds; the fastest lane width stays
    pre_rounds = r.round
    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
        r.run_async(1)
    r.sync()

    props = torch.cuda.get_device_properties(local)
    uuid = getattr(props, "uuid", None)
    uuid = ("GPU-" + str(uuid)) if uuid is not None and not str(uuid).startswith("GPU-") else uuid
    sampler = clock_sampler(uuid if uuid else None)
    events = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(args.steps)]
    s0 = r.stats()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    epoch0 = time.time()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()  # L2 flush, ordered before the step, outside its events
        one_step(events[i])
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop(epoch0, time.time())
    s1 = r.stats()
    step_ms = [a.elapsed_time(c) for a, _, c in events]
    sweep_ms = [a.elapsed_time(b) for a, b, _ in events]
    total_ms = sum(step_ms)
    flips = s1["flips"] - s0["flips"]

    # End to end through the public calls, on a second handle of the same seed
    # and the same rounds (warm-up, then the timed ones) with the same L2
    # flush before each: a step is rewl_run(handle, 1 round) -- which reads
    # the device status block back -- and then the result into a host
    # buffer: rewl_get_lng(partial) (copies walker 0's ln g of every window
    # and the visited masks to the host and joins them), or, while some
    # neighbouring windows share no visited bin yet, rewl_get_field(ln g of
    # every walker).
    import numpy as np

    r2 = REWL(*WL.rewl_args(p, args.seed + rank), spin_bits=p["spin_bits"], stream=stream)
    if args.schedule == "inv_t":
        r2.set_option(_lib.OPT_SCHEDULE, _lib.SCHEDULE_INV_T)
        r2.set("phase", 1)
    if pre_rounds:  # the rounds the autotuner ran on the first handle, in the chosen lane width
        r2.set_option(_lib.OPT_LANES, r.get_option(_lib.OPT_LANES))
        r2.run(pre_rounds)
    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
        r2.run_async(1)
    r2.sync()
    e2e_s, d2h, reads = 0.0, 0, {"rewl_get_lng": 0, "rewl_get_field": 0}
    e0s = r2.stats()["flips"]
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        t0 = time.perf_counter()
        r2.run(1)
        try:
            res = r2.lng(partial=True)
            d2h += 64 + p["h"] * r2.B * 9  # status, ln g rows and masks
            reads["rewl_get_lng"] += 1
        except RewlError:
            res = r2.get("lng")
            d2h += 64 + res.nbytes
            reads["rewl_get_field"] += 1
        e2e_s += time.perf_counter() - t0
    e2e_flips = r2.stats()["flips"] - e0s
    e2e_local = e2e_flips / e2e_s
    assert np.isfinite(res).any()
    total_ms_max, flips_all, e2e_val = reduce_over_ranks(dist, "cuda", total_ms, flips, e2e_local)
    value = flips_all / (total_ms_max / 1e3)

    # Roofline of the dominant kernel (the sweep): its proposals per launch /
    # its mean launch time, against the per-flip bound of each pipe (measured
    # issue rates x SMs x the SM clock sampled during the timed region /
    # algorithmic operations per flip of that pipe); the binding one is the
    # smallest.
    from paper_1312_3004_gb300 import measure_pipes

    pipes = measure_pipes()
    active_walkers = flips / max(1, args.steps) / p["exchange_interval"]
    sweep_avg_s = statistics.mean(sweep_ms) / 1e3
    achieved = active_walkers * p["exchange_interval"] / sweep_avg_s
    f_hz = (clocks.get("sm_mhz") or pipes["max_clock_mhz"]) * 1e6
    nsm = pipes["sms"]
    cpu = None
    if world == 1 and not args.no_cpu_baseline and args.workload != "potts10_L300":
        cpu = cpu_baseline(p, args.seed, args.cpu_seconds)
    rho = cpu["rho_neg"] if cpu else 0.0  # unknown: no exp charged (the higher bound)
    bounds = pipe_bounds(pipes, f_hz, rho)
    binding = min(bounds, key=bounds.get)
    # each walker's steps form one dependent chain: the clock cycles one step
    # of one walker takes, against the latency of the chain's shared-memory
    # load and integer add
    chain = active_walkers * f_hz / achieved if achieved > 0 else None

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    line = {
        "metric": "flip attempts/s", "value": value, "unit": "flips/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(config_of(args.workload, p), parallelism="replicas" if world > 1 else "single",
                                            lnf_schedule=args.schedule),
        "roofline": {"bound": binding, "achieved": achieved, "peak": bounds[binding], "unit": "flips/s",
                     "frac": achieved / bounds[binding],
                     # the ncu figures were taken on the halving schedule's fast sweep
                     "traffic": TRAFFIC_PER_LAUNCH.get(args.workload) if args.schedule == "halving" else None,
                     "kernel": "sweep_fast_kernel" if r.get_option(_lib.OPT_SWEEP_KERNEL) == 0 else "sweep_kernel",
                     "avg_launch_ms": sweep_avg_s * 1e3,
                     "bounds_flips_per_s": bounds,
                     "ops_per_flip": dict(OPS_PER_FLIP, fp64=FP64_PER_FLIP + FP64_PER_EXP * rho),
                     "rho_neg": rho if cpu else None,
                     "pipes_per_clk_sm": {k: pipes[k] for k in ("dadd", "imad", "imad_hi", "lop3", "iadd", "lds")},
                     "peak_basis": "measured issue rates (rewl_measure_pipes) x %d SMs x %.0f MHz (median SM clock "
                                   "sampled in the timed region) / algorithmic operations per flip" % (nsm, f_hz / 1e6),
                     "chain_cycles_per_step": chain,
                     "latency_cycles": {k: pipes[k] for k in ("dadd_latency", "imad_latency", "lds_latency")},
                     "walkers": active_walkers},
        "e2e": {"value": e2e_val, "unit": "flips/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": d2h / args.steps, "steps": args.steps, "reads": reads,
                "call": "rewl_run(handle, 1 round) + rewl_get_lng(partial) into a host buffer, per step, on a "
                        "second handle of the same seed over the same rounds, L2 flushed before each (untimed)"},
        "gpu_launches": 3 * args.steps,
        "sweep_plan": {"kernel": "fast" if r.get_option(_lib.OPT_SWEEP_KERNEL) == 0 else "reference",
                       "lanes_per_walker": r.get_option(_lib.OPT_LANES),
                       "walkers_per_cta": r.get_option(_lib.OPT_WALKERS_PER_CTA),
                       "lattice": "global" if r.get_option(_lib.OPT_LATTICE) else "shared"},
        "slow_path_decisions": r.stats()["slow_decisions"],
        "autotune": {"timed": tuned, "rounds_before_warmup": pre_rounds} if tuned is not None else None,
        "clocks": clocks,
        "wall_s_timed": wall,
        "sweep_share": sum(sweep_ms) / total_ms,
    }
    if cpu:
        line["cpu_baseline"] = cpu
    if args.workload == "potts10_L300":
        # the oracle's window entry alone (2151 walkers, most of them quenched
        # down to their windows one proposal at a time) outlasts the budget
        line["cpu_baseline"] = None
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
def run_batched(args):
    """2048 independent instances of uneven size in one batch vs the same kind
    of instances launched one at a time (plain form), same rounds."""
    import numpy as np
    import torch

    from paper_1312_3004_gb300 import REWL, Batch
    from paper_1312_3004_gb300 import workloads as WL

    jobs = WL.batched_instances(args.instances)
    stream = torch.cuda.Stream()

    # the batched form: created with the size rule, then the autotuner times its
    # candidate configurations on the first rounds (ordinary rounds of the run)
    # and keeps the fastest
    t0 = time.perf_counter()
    b = Batch(jobs)
    t_create = time.perf_counter() - t0
    b.set_stream(stream)
    t0 = time.perf_counter()
    tuned, cached = b.autotune(2)
    t_tune = time.perf_counter() - t0
    cfg = b.config()
    b.run_async(args.warmup)
    b.sync()
    f0 = b.stats()["flips"]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    props = torch.cuda.get_device_properties(0)
    uuid = getattr(props, "uuid", None)
    uuid = ("GPU-" + str(uuid)) if uuid is not None and not str(uuid).startswith("GPU-") else uuid
    sampler = clock_sampler(uuid)
    sampler.start()
    time.sleep(0.3)
    epoch0 = time.time()
    ev[0].record(stream)
    b.run_async(args.steps)
    ev[1].record(stream)
    b.sync()
    clocks = sampler.stop(epoch0, time.time())
    ms = ev[0].elapsed_time(ev[1])
    flips = b.stats()["flips"] - f0
    value = flips / (ms / 1e3)
    # plain: a sample of the instances, each alone, one after another
    rng = np.random.default_rng(7)
    sample = [jobs[i] for i in rng.choice(len(jobs), size=48, replace=False)]
    p_ms, p_flips = 0.0, 0
    for j in sample:
        r = REWL(*WL.rewl_args(j, j["seed"]), stream=stream)
        r.run_async(args.warmup)
        r.sync()
        f0 = r.stats()["flips"]
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r.run_async(args.steps)
        c.record(stream)
        r.sync()
        p_ms += a.elapsed_time(c)
        p_flips += r.stats()["flips"] - f0
        r.close()
    plain = p_flips / (p_ms / 1e3)
    info = b.info()
    from paper_1312_3004_gb300 import measure_pipes

    pipes = measure_pipes()
    f_hz = (clocks.get("sm_mhz") or pipes["max_clock_mhz"]) * 1e6
    bounds = pipe_bounds(pipes, f_hz, 0.0)  # no exp charged: the oracle is not run here
    binding = min(bounds, key=bounds.get)
    captured = args.instances == 2048 and cfg == {"spin_bits": 8, "lanes": 1, "cta_kb": 0, "threads": 128}
    line = {"metric": "flip attempts/s", "value": value, "unit": "flips/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batched2048" if args.instances == 2048 else "batched%d" % args.instances,
                       "instances": info["instances"], "walkers": info["walkers"],
                       "device_bytes": info["device_bytes"], "create_s": t_create,
                       "l2": "state larger than L2 (%.0f MB)" % (info["device_bytes"] / 1e6)},
            "plain": {"value": plain, "unit": "flips/s", "instances_sampled": len(sample),
                      "form": "one instance per launch, instances one after another"},
            "batched_over_plain": value / plain, "gpu_launches": 3 * args.steps,
            "autotune": {"chosen": cfg, "from_cache": cached, "seconds": t_tune, "timed": tuned,
                         "rounds_per_candidate": 2},
            "clocks": clocks,
            "roofline": {"bound": binding, "achieved": value, "peak": bounds[binding], "unit": "flips/s",
                         "frac": value / bounds[binding], "bounds_flips_per_s": bounds,
                         "traffic": TRAFFIC_PER_LAUNCH["batched2048"] if captured else None,
                         "peak_basis": "measured issue rates x %d SMs x %.0f MHz / algorithmic operations per flip "
                                       "(binary64: 2 adds, no exp charged)" % (pipes["sms"], f_hz / 1e6)}}
    print(json.dumps(line), flush=True)


def run_serving(args):
    """Poisson arrivals served by continuous batching vs the same jobs served
    one at a time in arrival order (plain form: latency from a FIFO schedule of
    the jobs' measured solo run times)."""
    import numpy as np
    import torch

    from paper_1312_3004_gb300 import REWL, Server
    from paper_1312_3004_gb300 import workloads as WL

    trace = WL.serving_trace(n=args.jobs)
    srv = Server(pool_bytes=2 << 30, max_jobs=512)
    ids = []
    t0 = time.perf_counter()
    k = 0
    while True:
        now = time.perf_counter() - t0
        while k < len(trace) and trace[k][0] <= now:
            ids.append((srv.submit(**trace[k][1]), trace[k][0]))
            k += 1
        running, queued = srv.step(rounds=4)
        if k == len(trace) and running == 0 and queued == 0:
            break
        if running == 0 and queued == 0 and k < len(trace):
            time.sleep(max(0.0, min(0.01, trace[k][0] - (time.perf_counter() - t0))))
    wall = time.perf_counter() - t0
    lat = []
    for jid, arrival in ids:
        info = srv.job_info(jid)
        lat.append(info["t_done"] - (t0 + arrival) if info["t_done"] > 0 else float("nan"))
    lat = np.array(lat)
    flips = srv.info()["flips"]
    # plain: every job alone, timed, then served first-come first-served
    solo = []
    for _, p in trace:
        r = REWL(*WL.rewl_args(p, p["seed"]))
        torch.cuda.synchronize()
        a = time.perf_counter()
        r.run(0)
        solo.append(time.perf_counter() - a)
        r.close()
    finish, plat = 0.0, []
    for (arrival, _), d in zip(trace, solo):
        finish = max(finish, arrival) + d
        plat.append(finish - arrival)
    plat = np.array(plat)
    line = {"metric": "request latency p50/p99", "value": float(np.percentile(lat, 99)), "unit": "s (p99)",
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "throughput_flips_per_s": flips / wall, "n_gpus": 1, "higher_is_better": False,
            "data": "synthetic", "jobs": len(trace), "arrival_rate_per_s": 50.0, "wall_s": wall,
            "config": {"workload": "serving", "trace": "Poisson 50/s, q 2..10, L 6..12, h 2..6, m 2..4, "
                                                       "ln f_final 1e-4/1e-5, K 2000 (trimmed to converge in seconds)"},
            "plain": {"p50_s": float(np.percentile(plat, 50)), "p99_s": float(np.percentile(plat, 99)),
                      "form": "each job alone, one at a time, first-come first-served",
                      "busy_s": float(sum(solo))}}
    print(json.dumps(line), flush=True)


def run_serving_full(args):
    """The serving workload at its stated sizes: the first --jobs arrivals of a
    Poisson stream (50/s) of jobs with q 2..10, L 16..96, h 8..64, m 2..8,
    ln f_final 1e-6 / 1e-8.  Calibration first: every job's cost is estimated
    (workloads.job_cost_estimate) and the offered load (estimated proposals per
    second of trace) is set against the server's measured capacity.  The full
    stream offers about a thousand times the capacity of one GPU, so it is
    trimmed by a cost cap (--cost-cap proposals): the jobs under the cap are
    served by continuous batching at their own arrival times, the others are
    left out and counted.  Plain form: each served job alone, one at a time in
    arrival order; its solo time is its own proposal count (the same alone as
    in the mix) over its solo rate, measured on the job alone over its first
    rounds (which overstates the solo rate late in a run: the plain latencies
    are a lower bound)."""
    import numpy as np
    import torch

    from paper_1312_3004_gb300 import REWL, Server
    from paper_1312_3004_gb300 import workloads as WL

    full = WL.serving_trace_full(n=args.jobs)
    span = full[-1][0]
    costs = [WL.job_cost_estimate(p) for _, p in full]
    kept = [(t, p, c) for (t, p), c in zip(full, costs) if c <= args.cost_cap]
    # capacity at full load: every served job resident at once, ~10 s of rounds
    cal = Server(pool_bytes=8 << 30, max_jobs=1024)
    for _, p, _ in kept:
        cal.submit(**p)
    cal.step(rounds=1)
    f0 = cal.info()["flips"]
    a = time.perf_counter()
    while time.perf_counter() - a < 10.0:
        cal.step(rounds=4)
    capacity_full = (cal.info()["flips"] - f0) / (time.perf_counter() - a)
    cal.close()
    srv = Server(pool_bytes=8 << 30, max_jobs=1024)
    ids = []
    t0 = time.perf_counter()
    k = 0
    busy_flips, busy_s = 0, 0.0
    while True:
        now = time.perf_counter() - t0
        while k < len(kept) and kept[k][0] <= now:
            ids.append((srv.submit(**kept[k][1]), kept[k][0], kept[k][2]))
            k += 1
        f_before = srv.info()["flips"]
        a = time.perf_counter()
        running, queued = srv.step(rounds=4)
        if running:
            busy_s += time.perf_counter() - a
            busy_flips += srv.info()["flips"] - f_before
        if k == len(kept) and running == 0 and queued == 0:
            break
        if running == 0 and queued == 0 and k < len(kept):
            time.sleep(max(0.0, min(0.01, kept[k][0] - (time.perf_counter() - t0))))
    wall = time.perf_counter() - t0
    lat, jflips = [], []
    for jid, arrival, _ in ids:
        info = srv.job_info(jid)
        lat.append(info["t_done"] - (t0 + arrival) if info["t_done"] > 0 else float("nan"))
        jflips.append(info["flips"])
    lat = np.array(lat)
    busy_rate = busy_flips / max(busy_s, 1e-9)
    # plain: each job alone, one at a time in arrival order
    solo = []
    stream = torch.cuda.Stream()
    for (_, p, _), fl in zip(kept, jflips):
        r = REWL(*WL.rewl_args(p, p["seed"]), stream=stream)
        r.run(1)
        f0 = r.stats()["flips"]
        torch.cuda.synchronize()
        a = time.perf_counter()
        r.run(4)
        dt = time.perf_counter() - a
        rate = (r.stats()["flips"] - f0) / dt if dt > 0 else float("inf")
        solo.append(fl / rate)
        r.close()
    finish, plat = 0.0, []
    for (arrival, _, _), d in zip(kept, solo):
        finish = max(finish, arrival) + d
        plat.append(finish - arrival)
    plat = np.array(plat)
    line = {"metric": "request latency p50/p99", "value": float(np.percentile(lat, 99)), "unit": "s (p99)",
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "throughput_flips_per_s": srv.info()["flips"] / wall, "n_gpus": 1, "higher_is_better": False,
            "data": "synthetic", "wall_s": wall,
            "config": {"workload": "serving_full", "arrivals": len(full), "arrival_rate_per_s": 50.0,
                       "trace": "Poisson 50/s, q 2..10, L 16..96, h 8..64, m 2..8, ln f_final 1e-6/1e-8, K 10^4"},
            "calibration": {"offered_flips_per_s_full": float(sum(costs) / span),
                            "capacity_flips_per_s": capacity_full,
                            "capacity_how": "every served job resident at once, 10 s of rounds",
                            "mean_rate_while_busy": busy_rate,
                            "offered_over_capacity_full": float(sum(costs) / span / capacity_full),
                            "cost_cap_proposals": args.cost_cap, "served_jobs": len(kept),
                            "left_out_jobs": len(full) - len(kept),
                            "offered_flips_per_s_served": float(sum(c for _, _, c in kept) / span),
                            "measured_over_estimated_cost": float(sum(jflips) / max(1.0, sum(c for _, _, c in kept))),
                            "cost_model": "workloads.job_cost_estimate"},
            "plain": {"p50_s": float(np.percentile(plat, 50)), "p99_s": float(np.percentile(plat, 99)),
                      "form": "each served job alone, one at a time, first-come first-served (solo time = its "
                              "proposals / its solo rate over its first rounds: a lower bound)",
                      "busy_s": float(sum(solo))}}
    print(json.dumps(line), flush=True)


def run_production(args):
    """Fixed-weight production (Sec. 3.2) on a named workload: --warmup WL
    rounds first (the walkers' ln g is then their estimate so far), then
    production with H(E, O) of the majority count in 64 classes; --steps
    production rounds are timed with events on the handle's stream."""
    import torch

    from paper_1312_3004_gb300 import REWL
    from paper_1312_3004_gb300 import workloads as WL

    p = WL.params(args.workload)
    stream = torch.cuda.Stream()
    r = REWL(*WL.rewl_args(p, args.seed), spin_bits=p["spin_bits"], stream=stream)
    r.run(max(1, args.warmup))
    r.production_start(64)
    r.production_run(1)
    f0 = r.stats()["flips"]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    r.production_run(args.steps)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    flips = r.stats()["flips"] - f0
    print(json.dumps({"metric": "production flip attempts/s", "value": flips / (ms / 1e3), "unit": "flips/s",
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                      "higher_is_better": True, "data": "synthetic", "gpu_launches": 2 * args.steps,
                      "config": dict(config_of(args.workload, p), production_classes=64),
                      "heo_total": int(r.heo().sum())}), flush=True)


def run_weak_scaling(args):
    """Time to convergence of several workloads run together, one stream
    each, one seed (the GPU analogue of Fig. 4's weak scaling: as N grows
    the number of windows grows, each window keeps its width, and the paper
    finds the time to a full density of states almost constant)."""
    import torch

    from paper_1312_3004_gb300 import REWL
    from paper_1312_3004_gb300 import workloads as WL

    names = [x for x in args.weak_scaling.split(",") if x]
    props = torch.cuda.get_device_properties(0)
    uuid = getattr(props, "uuid", None)
    uuid = ("GPU-" + str(uuid)) if uuid is not None and not str(uuid).startswith("GPU-") else uuid
    sampler = ClockSampler(uuid if uuid else None)
    sampler.start()
    epoch0 = time.time()
    hs = []
    for n in names:
        p = WL.params(n)
        hs.append((n, p, REWL(*WL.rewl_args(p, args.seed), spin_bits=p["spin_bits"], stream=torch.cuda.Stream())))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    finish, traces, el, last = {}, {n: [] for n in names}, 0.0, 0.0
    while len(finish) < len(hs) and el < args.converge_limit:
        for n, _, r in hs:
            if n not in finish:
                r.run_async(50)
        for n, _, r in hs:
            if n not in finish and r.sync():
                finish[n] = time.perf_counter() - t0
                print(json.dumps({"converged": n, "seconds": finish[n]}), flush=True)
        el = time.perf_counter() - t0
        if el - last >= 60.0:
            last = el
            for n, _, r in hs:
                st = r.stats()
                traces[n].append([round(el, 1), st["windows_done"], st["max_lnf"]])
            print(json.dumps({"progress_s": round(el, 1), "runs": {k: v[-1][1:] for k, v in traces.items() if v}}),
                  flush=True)
    clocks = sampler.stop(epoch0, time.time())
    runs = []
    for n, p, r in hs:
        st = r.stats()
        secs = finish.get(n, el)
        runs.append({"workload": n, "N": p["L"] ** 2, "windows": p["h"], "bins_per_window": r.W + 1,
                     "walkers": p["h"] * p["m"], "converged": n in finish, "seconds": secs, "rounds": st["rounds"],
                     "flips": st["flips"], "steps_per_walker": st["flips"] / (p["h"] * p["m"]),
                     "windows_done": st["windows_done"], "progress": traces[n],
                     "analysis": analyse(r, p) if n in finish else None})
        r.close()
    print(json.dumps({"metric": "time to converge, weak scaling", "unit": "s", "higher_is_better": False,
                      "n_gpus": 1, "data": "synthetic", "seed": args.seed, "limit_s": args.converge_limit,
                      "clocks": clocks, "runs": runs}), flush=True)


def analyse(r, p):
    """Canonical analysis of a converged run's joined ln g through the
    library: the specific-heat maximum and the equal-peak temperature Tc(L)
    with the suppression of the transition states (Sec. 3.1), searched within
    [0.8, 1.3] x the exact infinite-lattice Tc = 1 / ln(1 + sqrt(q))."""
    import math

    import paper_1312_3004_gb300 as P

    lng = r.lng()
    tc_inf = 1.0 / math.log(1.0 + math.sqrt(p["q"]))
    lo, hi = 0.8 * tc_inf, 1.3 * tc_inf
    T, c = P.specific_heat_peak(lng, lo, hi)
    out = {"T_range": [lo, hi], "c_peak_T": T, "c_peak": c, "Tc_equal_peak": None}
    try:
        Tc, a, b, sup = P.equal_peak_temperature(lng, lo, hi)
        out.update({"Tc_equal_peak": Tc, "E_peaks": [a, b], "log10_suppression": sup / math.log(10.0)})
    except P.RewlError:
        pass  # no double peak in the range (a continuous transition)
    return out


def oracle_reference(workload, seed, analysis, lng=None):
    """The oracle's converged values for this workload and seed, when stored
    (tests/golden/<workload>_converged.json, written by a script that runs
    only the oracle), with the oracle's mean and standard deviation over its
    seeds: the GPU run of the same seed reproduces the oracle's run, so its
    analysis must agree with the stored one."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", workload + "_converged.json")
    if analysis is None or not os.path.exists(path):
        return None
    with open(path) as f:
        ref = json.load(f)
    mine = [r for r in ref["runs"] if r["seed"] == seed]
    out = {"oracle_seeds": len(ref["runs"]), "oracle_mean": ref["mean"], "oracle_sd": ref["sd"]}
    if mine:
        r = mine[0]
        out["oracle_same_seed"] = {k: r[k] for k in ("c_peak_T", "c_peak", "Tc_equal_peak", "E_peaks")}
        out["same_as_oracle"] = (abs(analysis["c_peak_T"] - r["c_peak_T"]) <= 1e-6 * r["c_peak_T"] and
                                 abs(analysis["c_peak"] - r["c_peak"]) <= 1e-9 * r["c_peak"] and
                                 analysis.get("E_peaks") == r["E_peaks"])
    for key in ("c_peak_T", "c_peak", "Tc_equal_peak"):
        if analysis.get(key) is not None and ref["sd"].get(key) and ref["mean"].get(key) is not None:
            out.setdefault("sigmas_from_oracle_mean", {})[key] = (analysis[key] - ref["mean"][key]) / ref["sd"][key]
    if lng is not None and "lng_mean" in ref:
        # the run's normalised ln g against the oracle's seed mean, bin by bin, in
        # units of the oracle's single-run standard deviation
        z = [(x - m) / sd for x, m, sd in zip(lng, ref["lng_mean"], ref["lng_sd"]) if m is not None and sd > 0]
        out["lng_bins"] = len(z)
        out["lng_within_3sd"] = sum(abs(v) <= 3.0 for v in z) / max(1, len(z))
        out["lng_max_abs_z"] = max((abs(v) for v in z), default=None)
    return out


def run_converge(args):
    """Time to convergence (every window at ln f < ln f_final) of full runs,
    one per seed: wall time of rewl_run from the created handle (set-up and
    window entry included) until the status block reports convergence."""
    import torch

    from paper_1312_3004_gb300 import REWL
    from paper_1312_3004_gb300 import workloads as WL

    p = WL.params(args.workload)
    seeds = [int(x) for x in args.converge.split(",") if x.strip()]
    runs = []
    props = torch.cuda.get_device_properties(0)
    uuid = getattr(props, "uuid", None)
    uuid = ("GPU-" + str(uuid)) if uuid is not None and not str(uuid).startswith("GPU-") else uuid
    sampler = ClockSampler(uuid if uuid else None)
    sampler.start()
    epoch0 = time.time()
    if args.concurrent:
        # A run longer than one job of the machine is run in segments: the state of
        # every unfinished seed is saved (rewl_save) with the seconds it has run,
        # and the next segment loads it (rewl_load) and adds those seconds -- the
        # resumed run is the same run, step for step.
        prior, done_before, traces = {}, {}, {}
        for seed in seeds:
            meta = os.path.join(args.converge_resume, "seed%d.json" % seed) if args.converge_resume else None
            if meta and os.path.exists(meta):
                with open(meta) as f:
                    m = json.load(f)
                prior[seed] = m["seconds"]
                traces[seed] = m["progress"]
                if m["converged"]:
                    done_before[seed] = m
        hs = []
        for seed in seeds:
            if seed in done_before:
                continue
            r = REWL(*WL.rewl_args(p, seed), spin_bits=p["spin_bits"], stream=torch.cuda.Stream())
            if seed in prior:
                import zlib

                with open(os.path.join(args.converge_resume, "seed%d.blob" % seed), "rb") as f:
                    r.load(zlib.decompress(f.read()))
            hs.append((seed, r))
            traces.setdefault(seed, [])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        finish = {}
        el, last = 0.0, 0.0
        while len(finish) < len(hs) and el < args.converge_limit:
            for seed, r in hs:
                if seed not in finish:
                    r.run_async(50)
            for seed, r in hs:
                if seed not in finish and r.sync():
                    finish[seed] = time.perf_counter() - t0
                    print(json.dumps({"seed_converged": seed, "seconds": finish[seed]}), flush=True)
            el = time.perf_counter() - t0
            if el - last >= 60.0:  # progress: windows done and the largest ln f left
                last = el
                for seed, r in hs:
                    st = r.stats()
                    traces[seed].append([round(prior.get(seed, 0.0) + el, 1), st["windows_done"], st["max_lnf"]])
                print(json.dumps({"progress_s": round(el, 1), "seeds": {str(k): v[-1][1:] for k, v in traces.items()
                                                                         if v}}), flush=True)
        for seed, m in done_before.items():
            runs.append(m)
        for seed, r in hs:
            s = r.stats()
            secs = prior.get(seed, 0.0) + finish.get(seed, el)
            if args.converge_save and seed not in finish:
                os.makedirs(args.converge_save, exist_ok=True)
                import zlib

                with open(os.path.join(args.converge_save, "seed%d.blob" % seed), "wb") as f:
                    f.write(zlib.compress(r.save(), 1))
            runs.append({"seed": seed, "converged": seed in finish, "seconds": secs, "rounds": s["rounds"],
                         "flips": s["flips"], "mean_flips_per_s": s["flips"] / secs,
                         "windows_done": s["windows_done"], "progress": traces[seed],
                         "analysis": analyse(r, p) if seed in finish else None})
            runs[-1]["oracle"] = oracle_reference(args.workload, seed, runs[-1]["analysis"],
                                                  r.lng() if seed in finish else None)
            runs[-1]["segments"] = (1 + (1 if seed in prior else 0))
            if args.converge_save:
                os.makedirs(args.converge_save, exist_ok=True)
                with open(os.path.join(args.converge_save, "seed%d.json" % seed), "w") as f:
                    json.dump(runs[-1], f)
            r.close()
    for seed in ([] if args.concurrent else seeds):
        r = REWL(*WL.rewl_args(p, seed), spin_bits=p["spin_bits"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        conv, trace, last = False, [], 0.0
        while True:
            conv = r.run(200)
            el = time.perf_counter() - t0
            if conv or el > args.converge_limit:
                break
            if el - last >= 30.0:
                s = r.stats()
                trace.append([round(el, 1), s["windows_done"], s["max_lnf"]])
                last = el
        s = r.stats()
        runs.append({"seed": seed, "converged": bool(conv), "seconds": el, "rounds": s["rounds"],
                     "flips": s["flips"], "mean_flips_per_s": s["flips"] / el, "windows_done": s["windows_done"],
                     "progress": trace, "analysis": analyse(r, p) if conv else None})
        runs[-1]["oracle"] = oracle_reference(args.workload, seed, runs[-1]["analysis"], r.lng() if conv else None)
        print(json.dumps({"seed_done": runs[-1]}), flush=True)
        r.close()
    clocks = sampler.stop(epoch0, time.time())
    done = [x["seconds"] for x in runs if x["converged"]]
    line = {"metric": "time to converge", "clocks": clocks, "value": statistics.median(done) if len(done) == len(runs) else None,
            "unit": "s", "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
            "config": config_of(args.workload, p), "seeds": seeds,
            "min_s": min(done) if done else None, "max_s": max(done) if done else None,
            "limit_s": args.converge_limit, "concurrent": bool(args.concurrent), "runs": runs}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.converge:
        run_converge(args)
    elif args.production:
        run_production(args)
    elif args.weak_scaling:
        run_weak_scaling(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched2048":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "serving_full":
        run_serving_full(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
