"""The 1/t ln f schedule on the GPU against the oracle, bit for bit.

After the switch ln f = (bins in the mask) / (WL steps per walker) is not a
power of two, so every WL step of the fast sweep takes its binary64 add
(an integer step in the shadow's units cannot represent it); these tests run
through the switch and on to convergence in every sweep variant.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_3004_gb300 import REWL, RewlError
from paper_1312_3004_gb300 import _lib
from test_gpu_parity import assert_parity

pytestmark = pytest.mark.gpu

CASES = [
    # q, L, h, o, m, lnf_final, flatness, K, seed
    (3, 4, 3, 0.75, 2, 1e-4, 0.8, 700, 1),
    (10, 6, 4, 0.75, 2, 1e-4, 0.8, 2000, 5),
    (2, 8, 4, 0.75, 3, 1e-4, 0.8, 1000, 7),
]


def _pair(case):
    gpu, orc = REWL(*case), O.OracleREWL(*case)
    gpu.set_option(_lib.OPT_SCHEDULE, _lib.SCHEDULE_INV_T)
    orc.set_schedule(1)
    return gpu, orc


def _check(gpu, orc):
    assert_parity(gpu, orc)
    assert np.array_equal(gpu.get("phase"), orc.phase())


@pytest.mark.parametrize("variant", ["fast", "lanes1", "reference"])
@pytest.mark.parametrize("case", CASES)
def test_inv_t_schedule_matches_the_oracle_to_convergence(case, variant):
    gpu, orc = _pair(case)
    if variant == "lanes1":
        gpu.set_option(_lib.OPT_LANES, 1)
    elif variant == "reference":
        gpu.set_option(_lib.OPT_SWEEP_KERNEL, 1)
    assert gpu.get_option(_lib.OPT_SCHEDULE) == 1
    switched = False
    for _ in range(400):
        gpu.run(25)
        orc.run(25)
        _check(gpu, orc)
        switched = switched or bool(orc.phase().any())
        if orc.all_done():
            break
    assert switched and orc.all_done() and gpu.stats()["converged"]
    lnf = gpu.get("lnf")
    assert np.all(lnf < case[5])
    assert np.any(lnf != 2.0 ** np.round(np.log2(lnf)))  # ln f = 1/t, not a power of two
    a, b = gpu.lng(), orc.lng_joined()
    fin = np.isfinite(b)
    assert np.array_equal(np.isfinite(a), fin)
    assert np.max(np.abs(a[fin] - b[fin])) <= 1e-12


def test_inv_t_save_load_and_schedule_checks():
    case = CASES[0]
    gpu, orc = _pair(case)
    gpu.run(60)
    blob = gpu.save()
    gpu.run(60)
    other = REWL(*case)
    with pytest.raises(RewlError):
        other.load(blob)  # saved under the 1/t rule, the handle halves
    other.set_option(_lib.OPT_SCHEDULE, 1)
    other.load(blob)
    other.run(60)
    for k in ("lng", "hist", "lnf", "phase", "steps", "spins", "round"):
        assert np.array_equal(gpu.get(k), other.get(k)), k
    with pytest.raises(RewlError):
        gpu.set_option(_lib.OPT_SCHEDULE, 2)
    orc.run(120)
    _check(gpu, orc)
