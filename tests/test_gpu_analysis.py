"""Canonical analysis of densities of states the CUDA path produced.

The library's analysis calls applied to GPU runs must give what the oracle's
analysis gives on the oracle's runs of the same seeds (the runs agree bit for
bit), and physics the exact density of states fixes: the specific-heat
maximum of the 2D Ising torus L = 8 (the q = 2 workload, ln f_final = 1e-6),
and a double peak above the exact q = 10 transition temperature 1/ln(1+sqrt 10)
for a small 10-state lattice (Sec. 3.1: Tc(L) approaches it from above).
"""
import math

import numpy as np
import pytest

import paper_1312_3004_gb300 as P
from oracle import oracle as O
from oracle import thermo as TH
from paper_1312_3004_gb300 import REWL
from paper_1312_3004_gb300 import workloads as WL
from tie_trace import TracedPair

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_specific_heat_peak_of_converged_ising_L8(seed):
    p = WL.params("ising_L8")
    gpu = REWL(*WL.rewl_args(p, seed), spin_bits=p["spin_bits"])
    orc = O.OracleREWL(*WL.rewl_args(p, seed))
    assert gpu.run(0) and orc.run(0)
    T, c = P.specific_heat_peak(gpu.lng(), 0.8, 2.0)
    T_o, c_o = TH.specific_heat_peak(orc.lng_joined(), 0.8, 2.0)
    assert T == pytest.approx(T_o, rel=1e-6)
    assert c == pytest.approx(c_o, rel=1e-9)
    T_x, c_x = TH.specific_heat_peak(O.exact_lng(O.exact_counts_tm(2, 8)), 0.8, 2.0)
    assert abs(T - T_x) < 0.02
    assert abs(c / c_x - 1.0) < 0.03


@pytest.mark.parametrize("seed", [5, 6])
def test_equal_peak_temperature_of_a_small_potts10_run(seed):
    args = (10, 6, 4, 0.75, 2, 1e-4, 0.8, 2000, seed)
    # the oracle follows the run (any difference traced to a logged near tie)
    tp = TracedPair(lambda: REWL(*args), lambda: O.OracleREWL(*args))
    tp.run(0)
    gpu, orc = tp.test, tp.orc
    assert orc.all_done()
    got = P.equal_peak_temperature(gpu.lng(), 0.6, 0.9)
    ref = TH.equal_peak_temperature(orc.lng_joined(), 0.6, 0.9)
    assert got[1:3] == ref[1:3]
    assert got[0] == pytest.approx(ref[0], rel=1e-12)
    assert got[3] == pytest.approx(ref[3], abs=1e-9)
    Tc, e_low, e_high, ln_sup = got
    assert 1.0 / math.log(1.0 + math.sqrt(10.0)) < Tc < 0.8
    assert -72 <= e_low < e_high <= 0 and ln_sup < 0
    p = P.canonical_distribution(gpu.lng(), Tc)
    assert p[e_low + 72] == pytest.approx(1.0, abs=1e-9)
    assert p[e_high + 72] == pytest.approx(1.0, abs=1e-9)


def test_bootstrap_over_gpu_runs_matches_the_oracle():
    """Pieces of four GPU runs, resampled: the library and the oracle agree."""
    args = [(3, 5, 3, 0.75, 2, 1e-3, 0.8, 500, s) for s in (11, 12, 13, 14)]
    runs = [REWL(*a) for a in args]
    for r in runs:
        assert r.run(0)
    pieces = [r.window_pieces() for r in runs]
    e_lo, W = pieces[0][0], pieces[0][1]
    lw = np.stack([x[2] for x in pieces])
    mw = np.stack([x[3] for x in pieces])
    draws = np.random.default_rng(2).integers(0, 4, size=(16, 4))
    got = P.bootstrap(3, 5, e_lo, W, lw, mw, draws)
    ref = TH.bootstrap(3, 25, e_lo, W, lw, mw, draws)
    assert np.array_equal(np.isfinite(got), np.isfinite(ref))
    assert np.allclose(got[np.isfinite(got)], ref[np.isfinite(ref)], rtol=0, atol=1e-12)
    Tpk = np.array([P.specific_heat_peak(row, 0.5, 2.0)[0] for row in got])
    assert np.all(np.isfinite(Tpk)) and Tpk.std() >= 0.0
