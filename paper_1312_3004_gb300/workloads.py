"""Seeded synthetic workloads (parameter sets only; no REWL arithmetic).

The paper's Potts runs (Sec. 3.1) are defined by lattice parameters and seeds;
there is no dataset.  These named configurations are shared by the tests, the
benchmark and the CPU baseline.
"""
import math

import numpy as np

# Each entry: q, L, h, overlap, m, lnf_final, flatness, exchange_interval, spin_bits
CONFIGS = {
    # 2D Ising (q=2 Potts) L=8, 4 windows, 2 walkers, ln f 1 -> 1e-6, 8-bit spins
    "ising_L8": dict(q=2, L=8, h=4, overlap=0.75, m=2, lnf_final=1e-6, flatness=0.8,
                     exchange_interval=10_000, spin_bits=8),
    # 10-state Potts L=20, 8 windows, 4 walkers, ln f_final 1e-8
    "potts10_L20": dict(q=10, L=20, h=8, overlap=0.75, m=4, lnf_final=1e-8, flatness=0.8,
                        exchange_interval=10_000, spin_bits=8),
    # smaller sizes of the same layout: the finite-size series of Tc(L) (Sec. 3.1)
    "potts10_L8": dict(q=10, L=8, h=8, overlap=0.75, m=4, lnf_final=1e-8, flatness=0.8,
                       exchange_interval=10_000, spin_bits=8),
    "potts10_L12": dict(q=10, L=12, h=8, overlap=0.75, m=4, lnf_final=1e-8, flatness=0.8,
                        exchange_interval=10_000, spin_bits=8),
    "potts10_L16": dict(q=10, L=16, h=8, overlap=0.75, m=4, lnf_final=1e-8, flatness=0.8,
                        exchange_interval=10_000, spin_bits=8),
    # 10-state Potts L=80 (N=6400), 64 windows x 16 walkers = 1024 walkers, 4-bit spins
    "potts10_L80": dict(q=10, L=80, h=64, overlap=0.75, m=16, lnf_final=1e-8, flatness=0.8,
                        exchange_interval=10_000, spin_bits=4),
    # The paper's own run (Sec. 3.1): 10-state Potts L=300 (N=90000), 717 windows of
    # 1000 bins at 75% overlap, 3 walkers each (2151 walkers), 4-bit spins (45 KB lattices)
    "potts10_L300": dict(q=10, L=300, h=717, overlap=0.75, m=3, lnf_final=1e-8, flatness=0.8,
                         exchange_interval=10_000, spin_bits=4),
    # Weak scaling (Sec. 3.1, Fig. 4: the number of windows grows with N so that each
    # window keeps its width): 10-state Potts at L = 40 and 80 with windows of 291 + 1
    # bins, as the L=20 workload's, 4 walkers each
    "potts10_L40_w291": dict(q=10, L=40, h=41, overlap=0.75, m=4, lnf_final=1e-8, flatness=0.8,
                             exchange_interval=10_000, spin_bits=8),
    "potts10_L80_w291": dict(q=10, L=80, h=173, overlap=0.75, m=4, lnf_final=1e-8, flatness=0.8,
                             exchange_interval=10_000, spin_bits=4),
}


def params(name, **override):
    p = dict(CONFIGS[name])
    p.update(override)
    return p


def rewl_args(p, seed):
    """Positional arguments of REWL(...) / OracleREWL(...) for a config dict."""
    return (p["q"], p["L"], p["h"], p["overlap"], p["m"], p["lnf_final"], p["flatness"],
            p["exchange_interval"], seed)


def batched_instances(n=2048, master_seed=0x5EED0003):
    """Independent instances of uneven size: q in {2,4,8,10}, L in {8,12,...,48},
    h in {4,8,16}, m in {2,4}, overlap 0.75, ln f_final 1e-6, flatness 0.8."""
    rng = np.random.default_rng(master_seed)
    out = []
    for i in range(n):
        out.append(dict(q=int(rng.choice([2, 4, 8, 10])), L=int(rng.choice(np.arange(8, 49, 4))),
                        h=int(rng.choice([4, 8, 16])), overlap=0.75, m=int(rng.choice([2, 4])),
                        lnf_final=1e-6, flatness=0.8, exchange_interval=10_000,
                        seed=int(rng.integers(1, 2**63))))
    return out


def serving_trace(n=100, rate=50.0, master_seed=0x5EED0005):
    """Poisson arrivals (exponential gaps, mean 1/rate s) of density-of-states
    jobs, trimmed so that every job converges within seconds on one GPU:
    q in {2..10}, L in {6..12}, h in {2..6}, m in {2..4}, ln f_final in
    {1e-4, 1e-5}, 2000 steps between exchanges, overlap 0.75, flatness 0.8.
    Returns [(arrival_s, params)]."""
    rng = np.random.default_rng(master_seed)
    t = 0.0
    out = []
    for _ in range(n):
        t += float(rng.exponential(1.0 / rate))
        out.append((t, dict(q=int(rng.integers(2, 11)), L=int(rng.integers(6, 13)), h=int(rng.integers(2, 7)),
                            overlap=0.75, m=int(rng.integers(2, 5)),
                            lnf_final=float(rng.choice([1e-4, 1e-5])), flatness=0.8,
                            exchange_interval=2000, seed=int(rng.integers(1, 2**63)))))
    return out


def serving_trace_full(n=1000, rate=50.0, master_seed=0x5EED0005):
    """Poisson arrivals (exponential gaps, mean 1/rate s) of density-of-states
    jobs at the serving workload's stated sizes: q in {2..10}, L in {16..96},
    h in {8..64}, m in {2..8}, ln f_final in {1e-6, 1e-8}, 10^4 steps between
    exchanges, overlap 0.75, flatness 0.8.  Returns [(arrival_s, params)]."""
    rng = np.random.default_rng(master_seed)
    t = 0.0
    out = []
    for _ in range(n):
        t += float(rng.exponential(1.0 / rate))
        out.append((t, dict(q=int(rng.integers(2, 11)), L=int(rng.integers(16, 97)), h=int(rng.integers(8, 65)),
                            overlap=0.75, m=int(rng.integers(2, 9)),
                            lnf_final=float(rng.choice([1e-6, 1e-8])), flatness=0.8,
                            exchange_interval=10_000, seed=int(rng.integers(1, 2**63)))))
    return out


def job_cost_estimate(p):
    """Estimated WL proposals for a job to converge: walkers x steps per
    walker, with steps per walker = 1.9e7 (W / 47)^1.83 x (iterations / 27),
    W the bins per window and iterations = ceil(log2(1 / ln f_final)) + 1 --
    a fit to converged runs of q = 10, h = 8, m = 4 at L = 8, 12, 16, 20 and
    ln f_final = 1e-8 (W = 47 .. 291; 1.9e7 .. 5.3e8 steps per walker).  Used
    only to calibrate the offered load of a serving trace and to cap it; large
    lattices near a first-order transition take longer than it says."""
    N = p["L"] * p["L"]
    R = 2 * N
    W = min(R, math.ceil(R / (1.0 + (p["h"] - 1) * (1.0 - p["overlap"]))))
    iters = math.ceil(math.log2(1.0 / p["lnf_final"])) + 1
    return p["h"] * p["m"] * 1.9e7 * (W / 47.0) ** 1.83 * iters / 27.0
