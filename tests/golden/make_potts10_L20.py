"""Writes tests/golden/potts10_L20_converged.json: the oracle's converged runs
of the 10-state Potts L = 20 workload (8 windows, 75 % overlap, 4 walkers,
ln f_final = 1e-8, flatness 0.8, K = 10^4), seeds 1-16, and the canonical
analysis of each joined ln g (Sec. 3.1): the specific-heat maximum and the
equal-peak temperature Tc(L) with the suppression of the transition states,
searched within [0.8, 1.3] x 1/ln(1 + sqrt 10).

Calls only the oracle (oracle/) and the workload table.  Each run takes
15-20 minutes of one core; the seeds run in parallel processes (one per core
but one), so the whole script takes about an hour on 8 cores.

    python tests/golden/make_potts10_L20.py
"""
import json
import math
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
SEEDS = tuple(range(1, 17))


def one(seed):
    sys.path.insert(0, ROOT)
    import warnings

    from oracle import oracle as O
    from oracle import thermo as TH
    from paper_1312_3004_gb300 import workloads as WL

    warnings.simplefilter("ignore")
    p = WL.params("potts10_L20")
    o = O.OracleREWL(*WL.rewl_args(p, seed))
    t0 = time.time()
    assert o.run(0)
    secs = time.time() - t0
    lng = o.lng_joined()
    tc_inf = 1.0 / math.log(1.0 + math.sqrt(p["q"]))
    lo, hi = 0.8 * tc_inf, 1.3 * tc_inf
    T, c = TH.specific_heat_peak(lng, lo, hi)
    Tc, e_low, e_high, ln_sup = TH.equal_peak_temperature(lng, lo, hi)
    steps = int(o.t().sum())
    return {"seed": seed, "rounds": int(o.round), "wl_steps": steps, "oracle_seconds": round(secs, 1),
            "c_peak_T": T, "c_peak": c, "Tc_equal_peak": Tc, "E_peaks": [e_low, e_high],
            "ln_suppression": ln_sup}


def main():
    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, min(len(SEEDS), (os.cpu_count() or 2) - 1))) as pool:
        runs = pool.map(one, SEEDS, chunksize=1)
    out = {
        "source": "oracle/ (rewl_oracle.c, thermo.py); written by tests/golden/make_potts10_L20.py",
        "workload": "potts10_L20: q=10, L=20, h=8, overlap 0.75, m=4, ln f_final 1e-8, flatness 0.8, K=10^4",
        "T_range": "[0.8, 1.3] x 1/ln(1+sqrt(10))",
        "runs": runs,
    }
    for key in ("c_peak_T", "c_peak", "Tc_equal_peak", "ln_suppression"):
        v = [r[key] for r in runs]
        mean = sum(v) / len(v)
        sd = math.sqrt(sum((x - mean) ** 2 for x in v) / (len(v) - 1))
        out.setdefault("mean", {})[key] = mean
        out.setdefault("sd", {})[key] = sd
    with open(os.path.join(HERE, "potts10_L20_converged.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
