"""Writes tests/golden/<workload>_seed_lng.json: the oracle's joined,
normalised ln g of converged runs of a named Potts workload
(paper_1312_3004_gb300/workloads.py) for a few seeds, each value stored
exactly (float.hex), with the number of near-tie acceptance draws
(|u - exp(D)| < 1e-12) the oracle met on the way.  A GPU run of the same
seed must reproduce these values bit for bit (where the oracle met no near
tie, nothing else is possible).

Calls only the oracle (oracle/) and the workload table.  One process per
seed; a converged q = 10, L = 20 run takes 15-20 minutes of one core.

    python tests/golden/make_seed_lng.py --workload potts10_L20 --seeds 1,2
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def one(job):
    workload, seed = job
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from paper_1312_3004_gb300 import workloads as WL

    p = WL.params(workload)
    o = O.OracleREWL(*WL.rewl_args(p, seed))
    t0 = time.time()
    assert o.run(0)
    n_ties, _ = o.ties()
    return {"seed": seed, "rounds": int(o.round), "oracle_seconds": round(time.time() - t0, 1),
            "near_ties_1e-12": n_ties, "lng_hex": [float(x).hex() for x in o.lng_joined()]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="potts10_L20")
    ap.add_argument("--seeds", default="1,2")
    args = ap.parse_args()
    seeds = [int(s) for s in args.seeds.split(",")]
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(seeds)) as pool:
        runs = pool.map(one, [(args.workload, s) for s in seeds], chunksize=1)
    out = {"source": "oracle/ (rewl_oracle.c); written by tests/golden/make_seed_lng.py --workload %s --seeds %s"
                     % (args.workload, args.seeds),
           "workload": args.workload, "runs": runs}
    with open(os.path.join(HERE, args.workload + "_seed_lng.json"), "w") as f:
        json.dump(out, f)
        f.write("\n")


if __name__ == "__main__":
    main()
