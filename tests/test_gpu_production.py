"""The fixed-weight production run on the GPU (Sec. 3.2: configurations
sampled with weights 1/g(E) once g(E) is estimated, distributions H(E, O)
recorded; here O is the Potts majority count) against the oracle's
production run.

Counts are integers and every decision is the oracle's, so H(E, O) and the
whole state (spins, energies, replica ids, step counters, ln g, H) must agree
exactly after every set of rounds.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_3004_gb300 import REWL, RewlError
from tie_trace import differing, gpu_state, gpu_ties, oracle_state

pytestmark = pytest.mark.gpu


def assert_same(gpu, orc):
    diff = differing(gpu_state(gpu), oracle_state(orc))
    assert not diff, "state differs in %s (near ties logged by the library: %s)" % (diff, gpu_ties(gpu))
    assert np.array_equal(gpu.heo(), orc.heo())


@pytest.mark.parametrize("args,wl_rounds,n_obins,bits", [
    ((3, 5, 2, 0.75, 2, 1e-3, 0.8, 500, 3), 6, 4, 8),      # small: 2 windows, partial WL run
    ((10, 12, 4, 0.75, 3, 1e-3, 0.8, 2000, 5), 20, 16, 4),  # q = 10, 4-bit spins, m = 3
    ((2, 8, 4, 0.75, 2, 1e-6, 0.8, 10_000, 1), 0, 33, 8),   # L = 8 Ising workload, converged first
])
def test_production_matches_the_oracle(args, wl_rounds, n_obins, bits):
    gpu = REWL(*args, spin_bits=bits)
    orc = O.OracleREWL(*args)
    gpu.run(wl_rounds)
    orc.run(wl_rounds)
    assert not differing(gpu_state(gpu), oracle_state(orc))
    gpu.production_start(n_obins)
    orc.production_start(n_obins)
    assert_same(gpu, orc)
    for n in (1, 3, 8):
        gpu.production_run(n)
        orc.production_run(n)
        assert_same(gpu, orc)
    assert int(gpu.heo().sum()) == 12 * args[7] * gpu.G  # every step counted once
    assert np.all(gpu.get("hist") == 0)


def test_production_restart_and_refusals():
    args = (4, 6, 3, 0.75, 2, 1e-3, 0.8, 400, 9)
    gpu = REWL(*args)
    with pytest.raises(RewlError):
        gpu.production_run(1)  # not started
    gpu.run(3)
    N = 36
    with pytest.raises(RewlError):
        gpu.production_start(0)
    with pytest.raises(RewlError):
        gpu.production_start(N - (N + 3) // 4 + 2)
    gpu.production_start(5)
    gpu.production_run(2)
    assert gpu.heo().sum() > 0
    with pytest.raises(RewlError):
        gpu.run(1)
    with pytest.raises(RewlError):
        gpu.save()
    gpu.production_start(5)  # restart: histogram zeroed
    assert gpu.heo().sum() == 0
    gpu.production_run(1)
    assert int(gpu.heo().sum()) == 400 * gpu.G


def test_a_planted_near_tie_in_production_is_logged():
    """ln g set so that the first production step of one walker has exp(D)
    within 1e-16 of its draw: the production kernel's single-precision bracket
    cannot decide it, the exact binary64 path does and logs the near tie, and
    the oracle sees the same near tie; the states agree or differ by that one
    decision."""
    from tie_trace import gpu_ties, planted_near_tie

    args = (3, 5, 2, 0.75, 2, 1e-3, 0.8, 200, 11)
    for g in range(4):
        if planted_near_tie(O.OracleREWL(*args), 11, g):
            break
    else:
        pytest.skip("no walker's first proposal stays in its window")
    gpu, orc = REWL(*args), O.OracleREWL(*args)
    gpu.production_start(4)
    orc.production_start(4)
    planted_near_tie(orc, 11, g, setter=lambda lng: gpu.set("lng", lng))
    gpu.production_run(1)
    orc.production_run(1)
    n, log = gpu_ties(gpu)
    assert n >= 1 and (0, g, 0) in log
    _, seen = orc.ties()
    assert any(e[:3] == (0, g, 0) and e[3] < 1e-14 for e in seen)
    if differing(gpu_state(gpu), oracle_state(orc)):  # the two exps decided differently
        o2 = O.OracleREWL(*args)
        o2.production_start(4)
        planted_near_tie(o2, 11, g)
        o2.invert_decision(0, g, 0)
        o2.production_run(1)
        assert not differing(gpu_state(gpu), oracle_state(o2)) and np.array_equal(gpu.heo(), o2.heo())
    else:
        assert np.array_equal(gpu.heo(), orc.heo())
