"""Stored values: the numbers Sec. 3.1 of the paper prints (tests/golden/
paper_sec3_1.json, cited there), and exact densities of states of small
lattices written by tests/golden/make_exact_dos.py from the oracle alone."""
import json
import math
import os

from oracle import oracle as O
from paper_1312_3004_gb300 import workloads as WL

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_paper_geometry_and_workload():
    p = load("paper_sec3_1.json")
    e_lo, W = O.window_table(p["L"], p["windows"], p["overlap"])
    assert W == 1000  # 2N / (1 + 716 * 0.25) = 180000 / 180
    assert all(b - a == 250 for a, b in zip(e_lo, e_lo[1:]))
    assert e_lo[0] == -2 * p["L"] ** 2 and e_lo[-1] + W == 0
    w = WL.params("potts10_L300")
    assert (w["q"], w["L"], w["h"], w["overlap"], w["m"]) == (p["q"], p["L"], p["windows"], p["overlap"],
                                                               p["walkers_per_window"])
    assert abs(p["windows"] * p["walkers_per_window"] - p["walkers_about"]) < 200


def test_paper_temperatures_and_range():
    p = load("paper_sec3_1.json")
    exact = 1.0 / math.log(1.0 + math.sqrt(p["q"]))  # Potts units, E = -sum delta
    assert round(exact, 6) == p["Tc_exact"]
    assert abs(p["Tc_inf_extrapolated"] - exact) <= p["Tc_inf_extrapolated_error"]
    assert p["Tc_L300"] > exact  # the finite-size transition lies above Tc
    # ln g spans from ln q (ground state) to about N ln q: N log10 q decades
    decades = p["L"] ** 2 * math.log10(p["q"])
    assert 0.8 * p["dos_orders_of_magnitude_almost"] < decades < p["dos_orders_of_magnitude_almost"]


def test_stored_exact_densities_of_states():
    d = load("exact_dos_small.json")
    for key, t in d.items():
        if key.startswith("_"):
            continue
        q, L = t["q"], t["L"]
        N = L * L
        g = [int(c) for c in t["counts"]]
        assert len(g) == 2 * N + 1
        assert sum(g) == q ** N, key
        # low-energy counts by hand (k broken bonds): all equal; one odd spin;
        # an adjacent equal pair; an adjacent pair of two different values
        assert g[0] == q and g[1] == g[2] == g[3] == g[5] == 0, key
        assert g[4] == q * (q - 1) * N, key
        if L >= 4:
            assert g[6] == 2 * N * q * (q - 1), key
            assert g[7] == 2 * N * q * (q - 1) * (q - 2), key
        # the oracle still computes the same table
        again = O.exact_counts_brute(q, L) if key.startswith("brute") else O.exact_counts_tm(q, L)
        assert again == g, key
    # the two methods agree where both apply
    assert O.exact_counts_tm(2, 4) == [int(c) for c in d["brute_q2_L4"]["counts"]]
