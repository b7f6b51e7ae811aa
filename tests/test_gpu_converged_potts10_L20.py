"""The 10-state Potts L = 20 workload (8 windows of 4 walkers, ln f_final =
1e-8) run to convergence on the GPU, two seeds at once on two streams, against
the oracle's stored converged runs of the same seeds.

The oracle met no near-tie draw in those runs (stored count), so the GPU's
joined, normalised ln g must equal the oracle's bit for bit; its canonical
analysis (Sec. 3.1, Fig. 3b: the specific-heat maximum and the equal-peak
temperature Tc(L)) then equals the oracle's stored one, and lies within the
spread of the oracle's 16 seeds.  About five minutes on a GB300.
"""
import json
import math
import os

import numpy as np
import pytest

import paper_1312_3004_gb300 as P
from paper_1312_3004_gb300 import REWL
from paper_1312_3004_gb300 import workloads as WL

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_two_seeds_converge_to_the_oracles_density_of_states():
    import torch

    with open(os.path.join(GOLDEN, "potts10_L20_seed_lng.json")) as f:
        stored = {r["seed"]: r for r in json.load(f)["runs"]}
    with open(os.path.join(GOLDEN, "potts10_L20_converged.json")) as f:
        summary = json.load(f)
    p = WL.params("potts10_L20")
    seeds = sorted(stored)[:2]
    runs = {s: REWL(*WL.rewl_args(p, s), spin_bits=p["spin_bits"], stream=torch.cuda.Stream()) for s in seeds}
    done = set()
    for _ in range(4000):  # 50 rounds per call; the runs need 1.2e5 - 1.6e5 rounds
        for s, r in runs.items():
            if s not in done:
                r.run_async(50)
        for s, r in runs.items():
            if s not in done and r.sync():
                done.add(s)
        if len(done) == len(runs):
            break
    assert done == set(seeds)
    tc_inf = 1.0 / math.log(1.0 + math.sqrt(p["q"]))
    for s, r in runs.items():
        ref = stored[s]
        assert ref["near_ties_1e-12"] == 0
        assert r.stats()["near_ties"] == 0
        assert r.round == ref["rounds"]
        want = np.array([float.fromhex(x) for x in ref["lng_hex"]])
        got = r.lng()
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
        T, c = P.specific_heat_peak(got, 0.8 * tc_inf, 1.3 * tc_inf)
        mine = [x for x in summary["runs"] if x["seed"] == s][0]
        assert T == pytest.approx(mine["c_peak_T"], rel=1e-9)
        assert c == pytest.approx(mine["c_peak"], rel=1e-9)
        for key, val in (("c_peak_T", T), ("c_peak", c)):
            assert abs(val - summary["mean"][key]) < 3 * summary["sd"][key]
        Tc, e_lo, e_hi, _ = P.equal_peak_temperature(got, 0.8 * tc_inf, 1.3 * tc_inf)
        assert [e_lo, e_hi] == mine["E_peaks"]
        assert tc_inf < Tc < T + 1e-3
