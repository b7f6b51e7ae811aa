"""Writes tests/golden/<workload>_converged.json: the oracle's converged runs
of a named Potts workload (paper_1312_3004_gb300/workloads.py) for a
range of seeds, and the canonical analysis of each joined ln g (Sec. 3.1): the
specific-heat maximum, the equal-peak temperature Tc(L) and the suppression of
the transition states, searched within [0.8, 1.3] x 1/ln(1 + sqrt q); with the
mean and sample standard deviation over the seeds of those numbers and of the
joined, normalised ln g bin by bin (lng_mean, lng_sd; null where no
configuration has that energy).

Calls only the oracle (oracle/) and the workload table.  The seeds run in
parallel processes, one per core but one.  A converged q = 10 run takes about
1 minute of one core at L = 8 and 15-20 minutes at L = 20.

    python tests/golden/make_converged.py                       # potts10_L20, seeds 1-16
    python tests/golden/make_converged.py --workload potts10_L12 --seeds 1-8
"""
import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def one(job):
    workload, seed = job
    sys.path.insert(0, ROOT)
    import warnings

    from oracle import oracle as O
    from oracle import thermo as TH
    from paper_1312_3004_gb300 import workloads as WL

    warnings.simplefilter("ignore")
    p = WL.params(workload)
    o = O.OracleREWL(*WL.rewl_args(p, seed))
    t0 = time.time()
    assert o.run(0)
    secs = time.time() - t0
    lng = o.lng_joined()
    tc_inf = 1.0 / math.log(1.0 + math.sqrt(p["q"]))
    lo, hi = 0.8 * tc_inf, 1.3 * tc_inf
    T, c = TH.specific_heat_peak(lng, lo, hi)
    peaks = TH.equal_peak_temperature(lng, lo, hi)   # None: no double peak (q = 2)
    Tc, e_low, e_high, ln_sup = peaks if peaks is not None else (None, None, None, None)
    steps = int(o.t().sum())
    return {"lng": [float(x) for x in lng], "seed": seed, "rounds": int(o.round), "wl_steps": steps, "oracle_seconds": round(secs, 1),
            "c_peak_T": T, "c_peak": c, "Tc_equal_peak": Tc,
            "E_peaks": [e_low, e_high] if e_low is not None else None,
            "ln_suppression": ln_sup}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="potts10_L20")
    ap.add_argument("--seeds", default="1-16", help="first-last")
    ap.add_argument("--procs", type=int, default=0, help="worker processes (0: one per core but one)")
    args = ap.parse_args()
    first, last = (int(x) for x in args.seeds.split("-"))
    seeds = list(range(first, last + 1))
    sys.path.insert(0, ROOT)
    from paper_1312_3004_gb300 import workloads as WL

    p = WL.params(args.workload)
    ctx = mp.get_context("spawn")
    procs = args.procs if args.procs > 0 else max(1, (os.cpu_count() or 2) - 1)
    with ctx.Pool(min(len(seeds), procs)) as pool:
        runs = pool.map(one, [(args.workload, s) for s in seeds], chunksize=1)
    out = {
        "source": "oracle/ (rewl_oracle.c, thermo.py); written by tests/golden/make_converged.py "
                  "--workload %s --seeds %s" % (args.workload, args.seeds),
        "workload": "%s: q=%d, L=%d, h=%d, overlap %g, m=%d, ln f_final %g, flatness %g, K=%d" % (
            args.workload, p["q"], p["L"], p["h"], p["overlap"], p["m"], p["lnf_final"], p["flatness"],
            p["exchange_interval"]),
        "T_range": "[0.8, 1.3] x 1/ln(1+sqrt(q))",
        "runs": runs,
    }
    lngs = [r.pop("lng") for r in runs]
    mean_b, sd_b = [], []
    for b in range(len(lngs[0])):
        v = [l[b] for l in lngs]
        if any(math.isinf(x) for x in v):
            assert all(math.isinf(x) for x in v)  # every run has the same support
            mean_b.append(None)
            sd_b.append(None)
            continue
        mu = sum(v) / len(v)
        mean_b.append(mu)
        sd_b.append(math.sqrt(sum((x - mu) ** 2 for x in v) / (len(v) - 1)) if len(v) > 1 else 0.0)
    out["lng_mean"] = mean_b
    out["lng_sd"] = sd_b
    for key in ("c_peak_T", "c_peak", "Tc_equal_peak", "ln_suppression"):
        v = [r[key] for r in runs if r[key] is not None]
        if len(v) < len(runs):
            out.setdefault("mean", {})[key] = None
            out.setdefault("sd", {})[key] = None
            continue
        mean = sum(v) / len(v)
        sd = math.sqrt(sum((x - mean) ** 2 for x in v) / (len(v) - 1)) if len(v) > 1 else 0.0
        out.setdefault("mean", {})[key] = mean
        out.setdefault("sd", {})[key] = sd
    with open(os.path.join(HERE, args.workload + "_converged.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
