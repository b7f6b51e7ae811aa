"""Pins of the oracle's fixed-weight production run (sampling with weights
1/g(E) after g(E) is known, measuring H(E,O); Sec. 3.2) and of the canonical
reweighting of its H(E,O) (oracle/thermo.py).

The observable is the Potts majority count n_max.  The exact microcanonical
distribution P(n_max | E) and the canonical <n_max>(T) come from enumerating
every configuration of small tori with numpy (energies and counts computed
here, independent of the oracle's code).
"""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import thermo as TH

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _enumerate(q, L):
    """(E, n_max) of every configuration of the periodic L x L torus."""
    N = L * L
    codes = np.arange(q ** N, dtype=np.int64)
    s = np.empty((q ** N, L, L), dtype=np.int8)
    for k in range(N):
        s[:, k // L, k % L] = codes % q
        codes //= q
    E = -((s == np.roll(s, 1, axis=1)).sum(axis=(1, 2)) + (s == np.roll(s, 1, axis=2)).sum(axis=(1, 2)))
    n_max = np.stack([(s == k).sum(axis=(1, 2)) for k in range(q)], axis=1).max(axis=1)
    return E, n_max


def _exact_heo(q, L):
    N = L * L
    E, n_max = _enumerate(q, L)
    lo = (N + q - 1) // q
    out = np.zeros((2 * N + 1, N - lo + 1))
    np.add.at(out, (E + 2 * N, n_max - lo), 1)
    return out


def _production(q, L, h, m, K, rounds, n_obins, seed=1):
    """A run whose walkers hold the exact ln g of their windows, then production."""
    N = L * L
    lng = O.exact_lng(O.exact_counts_tm(q, L))
    o = O.OracleREWL(q, L, h, 0.75, m, 1e-3, 0.8, K, seed)
    e_lo, W = o.e_lo(), o.W
    lw = np.zeros((h * m, W + 1))
    for w in range(h):
        seg = lng[e_lo[w] + 2 * N:e_lo[w] + 2 * N + W + 1]
        for k in range(m):
            lw[w * m + k] = np.where(np.isfinite(seg), seg, 0.0)
    o.set_lng(lw)
    o.production_start(n_obins)
    o.production_run(rounds)
    return o, lng


def test_majority_count_and_classes_by_hand():
    assert O.majority(np.array([0, 1, 1, 2, 1, 0, 2, 2, 2]), 3) == 4
    assert O.majority(np.zeros(16), 2) == 16
    # N = 9, q = 3: n_max in [3, 9]; 7 classes are the values, 2 classes split at 7
    assert [O.obin(n, 9, 3, 7) for n in range(3, 10)] == list(range(7))
    assert [O.obin(n, 9, 3, 2) for n in range(3, 10)] == [0, 0, 0, 0, 1, 1, 1]
    o = O.OracleREWL(3, 3, 1, 0.75, 1, 1e-3, 0.8, 10, 1)
    with pytest.raises(ValueError):
        o.production_start(8)
    with pytest.raises(ValueError):
        o.production_start(0)


@pytest.mark.parametrize("q,L,h", [(3, 3, 2), (2, 4, 3)])
def test_production_reproduces_the_exact_microcanonical_distribution(q, L, h):
    N = L * L
    n_o = N - (N + q - 1) // q + 1
    o, _ = _production(q, L, h, 2, 1000, 1500, n_o)
    C = TH.combine_heo(o.heo(), o.e_lo(), N).astype(float)
    X = _exact_heo(q, L)
    tot = C.sum(axis=1)
    assert np.array_equal(tot > 0, X.sum(axis=1) > 0)     # exactly the energies that exist
    ok = tot > 0
    P = C[ok] / tot[ok, None]
    Px = X[ok] / X[ok].sum(axis=1, keepdims=True)
    assert np.abs(P - Px).max() < 0.01
    assert np.array_equal(P > 0, Px > 0)                   # no impossible (E, O) pair sampled


def test_every_step_is_counted_once_and_ln_g_does_not_move():
    q, L, h, m, K, R = 3, 3, 2, 2, 700, 40
    o, _ = _production(q, L, h, m, K, 0, 7)
    before = o.lng().copy()
    o.production_run(R)
    assert int(o.heo().sum()) == h * m * K * R
    assert np.array_equal(o.lng().view(np.uint64), before.view(np.uint64))
    assert o.round == R


def test_fixed_weight_energy_marginal_is_flat():
    """With the exact g(E), weights 1/g(E) visit every energy of a window
    equally often (the multicanonical identity)."""
    o, _ = _production(2, 4, 2, 2, 1000, 1500, 9)
    for w in range(2):
        v = o.heo()[w].sum(axis=1).astype(float)
        v = v[v > 0]
        assert v.min() > 0.9 * v.mean() and v.max() < 1.1 * v.mean()


def test_coarse_classes_are_sums_of_fine_ones():
    """The class of O does not steer the sampling: the same seed gives the same
    trajectory, and coarse counts are the fine counts merged by the class map."""
    fine, _ = _production(3, 3, 2, 2, 500, 30, 7)
    coarse, _ = _production(3, 3, 2, 2, 500, 30, 2)
    f, c = fine.heo(), coarse.heo()
    merged = np.zeros_like(c)
    for v in range(7):
        merged[:, :, O.obin(3 + v, 9, 3, 2)] += f[:, :, v]
    assert np.array_equal(merged, c)


def test_canonical_observable_equals_the_sum_over_configurations():
    """<n_max>(T) from ln g and the exact P(n_max | E) equals the Boltzmann
    average over every configuration."""
    q, L = 3, 3
    N = L * L
    E, n_max = _enumerate(q, L)
    lng = O.exact_lng(O.exact_counts_brute(q, L))
    X = _exact_heo(q, L)
    lo = (N + q - 1) // q
    Ts = np.array([0.4, 0.8, 1.3, 3.0])
    got = TH.canonical_observable(lng, X, np.arange(lo, N + 1), Ts)
    for t, g in zip(Ts, got):
        w = np.exp(-(E - E.min()) / t)
        assert g == pytest.approx((w * n_max).sum() / w.sum(), rel=1e-12)


def test_canonical_observable_from_a_production_run():
    q, L = 3, 3
    N = L * L
    E, n_max = _enumerate(q, L)
    o, lng = _production(q, L, 2, 2, 1000, 1500, 7)
    C = TH.combine_heo(o.heo(), o.e_lo(), N)
    for t in (0.5, 1.0, 2.0):
        w = np.exp(-(E - E.min()) / t)
        exact = (w * n_max).sum() / w.sum()
        assert TH.canonical_observable(lng, C, np.arange(3, 10), [t])[0] == pytest.approx(exact, abs=0.01)
