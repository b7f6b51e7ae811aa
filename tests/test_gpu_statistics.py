"""GPU runs against the oracle's 16-seed statistics of the L=8 Ising workload
(tests/golden/ising_L8_converged.json, written by the oracle alone): a run of
a seed outside the oracle's 16 lies within 3 sigma of the oracle's per-bin mean
in nearly every bin (the reading of "within 3 sigma per energy bin" with
correlated bins), and its normalised ln g is within 0.35 of the exact one."""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_3004_gb300 import REWL
from paper_1312_3004_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("seed", [17, 18, 19, 20])
def test_gpu_run_within_3_sigma_of_the_oracle_mean(seed):
    with open(os.path.join(GOLDEN, "ising_L8_converged.json")) as f:
        d = json.load(f)
    mean = np.array([np.nan if m is None else m for m in d["lng_mean"]])
    sd = np.array([np.nan if v is None else v for v in d["lng_sd"]])
    ok = np.isfinite(mean)
    p = WL.params("ising_L8")
    r = REWL(*WL.rewl_args(p, seed), spin_bits=p["spin_bits"])
    assert r.run(0)
    lng = r.lng()
    assert np.array_equal(np.isfinite(lng), ok)
    z = (lng[ok] - mean[ok]) / sd[ok]
    assert np.mean(np.abs(z) <= 3.0) >= 0.9 and np.max(np.abs(z)) < 6.0
    exact = O.exact_lng(O.exact_counts_tm(2, 8))
    exact = exact - (np.logaddexp.reduce(exact[ok]) - 64 * np.log(2.0))
    assert np.max(np.abs(lng[ok] - exact[ok])) < 0.35
