"""Stored values: the numbers Sec. 3.1 of the paper prints (tests/golden/
paper_sec3_1.json, cited there), and exact densities of states of small
lattices written by tests/golden/make_exact_dos.py from the oracle alone."""
import json
import math
import os

import pytest

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


TC_Q10 = 1.0 / math.log(1.0 + math.sqrt(10.0))


def _check_converged_file(name, seeds):
    d = load(name + "_converged.json")
    runs = d["runs"]
    assert [r["seed"] for r in runs] == list(seeds)
    for key in ("c_peak_T", "c_peak", "Tc_equal_peak", "ln_suppression"):
        v = [r[key] for r in runs]
        mean = sum(v) / len(v)
        sd = math.sqrt(sum((x - mean) ** 2 for x in v) / (len(v) - 1))
        assert math.isclose(d["mean"][key], mean, rel_tol=1e-12)
        assert math.isclose(d["sd"][key], sd, rel_tol=1e-9, abs_tol=1e-300)
    p = WL.params(name)
    N = p["L"] ** 2
    assert len(d["lng_mean"]) == len(d["lng_sd"]) == 2 * N + 1
    # the support is the set of energies that exist: none of 1, 2, 3, 5 broken bonds
    assert [d["lng_mean"][k] is None for k in range(8)] == [False, True, True, True, False, True, False, False]
    # normalised: ln g(ground) = ln q up to the run-to-run error, sum g = q^N
    assert abs(d["lng_mean"][0] - math.log(p["q"])) < 5 * d["lng_sd"][0] + 0.05
    top = max(x for x in d["lng_mean"] if x is not None)
    s = sum(math.exp(x - top) for x in d["lng_mean"] if x is not None)
    assert abs(top + math.log(s) - N * math.log(p["q"])) < 0.05
    for r in runs:
        assert TC_Q10 < r["Tc_equal_peak"] < TC_Q10 + 0.08
        assert r["ln_suppression"] < 0
        assert -2 * N <= r["E_peaks"][0] < r["E_peaks"][1] <= 0
    return d


def test_converged_oracle_values_potts10_L20():
    """16 converged oracle runs of the q=10 L=20 workload (written by
    tests/golden/make_converged.py): the canonical analysis of each, and the
    per-bin mean and spread of ln g, are consistent."""
    d = _check_converged_file("potts10_L20", range(1, 17))
    for r in d["runs"]:
        assert abs(r["c_peak_T"] - r["Tc_equal_peak"]) < 0.002


def test_tc_of_L_approaches_the_exact_value_from_above():
    """Sec. 3.1: the finite-size transition temperature lies above
    1/ln(1 + sqrt 10), falls as L grows, and a fit Tc(L) = Tc + b/N over the
    oracle's L = 8 ... 20 runs extrapolates to the exact value within 1e-3
    (the paper extrapolates from L up to 300 to within 2e-6; at these sizes
    corrections beyond 1/N remain)."""
    series = []
    for L, seeds in ((8, range(1, 9)), (12, range(1, 9)), (16, range(1, 9)), (20, range(1, 17))):
        d = _check_converged_file("potts10_L%d" % L, seeds)
        n = len(d["runs"])
        series.append((L * L, d["mean"]["Tc_equal_peak"], d["sd"]["Tc_equal_peak"] / math.sqrt(n)))
    for (_, t0, e0), (_, t1, e1) in zip(series, series[1:]):
        assert t1 < t0 - 3 * math.hypot(e0, e1)     # decreasing with L, beyond the standard errors
    assert all(t > TC_Q10 for _, t, _ in series)
    # weighted least squares for Tc(L) = a + b / N
    w = [1.0 / e ** 2 for _, _, e in series]
    x = [1.0 / N for N, _, _ in series]
    y = [t for _, t, _ in series]
    sw = sum(w)
    xm = sum(wi * xi for wi, xi in zip(w, x)) / sw
    ym = sum(wi * yi for wi, yi in zip(w, y)) / sw
    b = sum(wi * (xi - xm) * (yi - ym) for wi, xi, yi in zip(w, x, y)) / sum(wi * (xi - xm) ** 2 for wi, xi in zip(w, x))
    a = ym - b * xm
    assert b > 0
    assert abs(a - TC_Q10) < 1e-3


def test_single_runs_lie_within_3_sigma_of_the_16_seed_mean_ising_L8():
    """The q=2 L=8 workload: 16 converged oracle runs give the per-bin mean and
    spread of ln g (tests/golden/ising_L8_converged.json); runs of other seeds
    fall within 3 sigma of that mean in nearly every bin, and the mean
    specific-heat peak lies within 3 standard errors of the exact torus's."""
    import numpy as np
    from oracle import thermo as TH

    d = load("ising_L8_converged.json")
    assert [r["seed"] for r in d["runs"]] == list(range(1, 17))
    mean = np.array([np.nan if m is None else m for m in d["lng_mean"]])
    sd = np.array([np.nan if v is None else v for v in d["lng_sd"]])
    ok = np.isfinite(mean)
    exact = O.exact_lng(O.exact_counts_tm(2, 8))
    assert np.array_equal(ok, np.isfinite(exact))          # the support: even k except 2 and 126
    p = WL.params("ising_L8")
    for seed in (17, 18, 19, 20):
        o = O.OracleREWL(*WL.rewl_args(p, seed))
        assert o.run(0)
        z = (o.lng_joined()[ok] - mean[ok]) / sd[ok]
        assert np.mean(np.abs(z) <= 3.0) >= 0.9 and np.max(np.abs(z)) < 6.0, seed
    T_x, c_x = TH.specific_heat_peak(exact, 0.8, 2.0)
    se = d["sd"]["c_peak_T"] / 4.0
    assert abs(d["mean"]["c_peak_T"] - T_x) < 3 * se


def test_stored_single_seed_runs_potts10_L20():
    """tests/golden/potts10_L20_seed_lng.json (written by make_seed_lng.py
    from the oracle alone): the exact joined ln g of seeds 1 and 2 is the
    oracle's run summarised in potts10_L20_converged.json -- the same rounds,
    the same support as the seed mean, sum g = q^N, ln g(ground) = ln q within
    the spread, and the same specific-heat maximum."""
    import numpy as np

    from oracle import thermo as TH

    seeds = load("potts10_L20_seed_lng.json")
    summary = load("potts10_L20_converged.json")
    N, q = 400, 10
    tc_inf = 1.0 / math.log(1.0 + math.sqrt(q))
    for run in seeds["runs"]:
        mine = [r for r in summary["runs"] if r["seed"] == run["seed"]][0]
        assert run["rounds"] == mine["rounds"]
        lng = np.array([float.fromhex(x) for x in run["lng_hex"]])
        fin = np.isfinite(lng)
        assert np.array_equal(fin, np.array([m is not None for m in summary["lng_mean"]]))
        top = lng[fin].max()
        assert abs(top + math.log(np.exp(lng[fin] - top).sum()) - N * math.log(q)) < 1e-9
        assert abs(lng[0] - math.log(q)) < 3 * summary["lng_sd"][0]
        T, c = TH.specific_heat_peak(lng, 0.8 * tc_inf, 1.3 * tc_inf)
        assert T == pytest.approx(mine["c_peak_T"], rel=1e-9)
        assert c == pytest.approx(mine["c_peak"], rel=1e-9)
