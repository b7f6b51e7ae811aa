"""Pins of the oracle's exchange pairing (Sec. 2: walker i picks its swap
partner j in a neighbouring window at random).

The reading: in a round, walker k of window a meets walker pi(k) of window
a + 1, pi a uniformly random permutation of the m walkers (a one-to-one
matching, so that each walker makes at most one exchange per round).  The
permutation is read back from the replica ids with every swap accepted (flat
ln g, so D = 0 in Eq. 1, and every energy inside both windows), and must be
uniform over all m! permutations -- a slip such as Sattolo's variant of the
shuffle (only cyclic permutations) or one random word reused for every swap
fails this -- independent between the window pairs of one round and between
rounds.
"""
import math
from collections import Counter
from itertools import permutations

import numpy as np
import pytest

from oracle import oracle as O


def chi2_sf(x, dof):
    """Survival function of the chi-square distribution (regularised upper
    incomplete gamma Q(dof/2, x/2), by its series / continued fraction)."""
    from scipy.special import gammaincc

    return float(gammaincc(dof / 2.0, x / 2.0))


def matching_fixture(m, h, seed):
    """An oracle instance whose walkers all carry one configuration with an
    energy inside every window's range (q = 3, L = 5: windows [-50, -10] and
    [-40, 0] for h = 2) and flat ln g, so that every exchange is accepted."""
    o = O.OracleREWL(3, 5, h, 0.75, m, 1e-3, 0.8, 100, seed)
    e_lo = o.e_lo()
    lo, hi = int(e_lo.max()), int(e_lo.min()) + o.W
    rng = np.random.default_rng(seed)
    while True:
        s = rng.integers(0, 3, o.N).astype(np.uint8)
        if lo <= O.energy(o.L, s) <= hi:
            break
    for g in range(o.G):
        o.set_config(g, s)
    o.set_lng(np.zeros((o.G, o.B)))
    return o


def matchings(o, r):
    """pi for every window pair (a, a+1) with a = r mod 2 in round r."""
    m = o.m
    before = o.rep()
    o.set_round(r)
    o.exchange()
    after = o.rep()
    out = {}
    for a in range(r % 2, o.h - 1, 2):
        pos = {int(before[(a + 1) * m + j]): j for j in range(m)}
        pi = tuple(pos[int(after[a * m + k])] for k in range(m))
        assert sorted(pi) == list(range(m))  # one-to-one
        out[a] = pi
    return out


@pytest.mark.parametrize("m,rounds", [(2, 4000), (3, 6000), (4, 12000)])
def test_every_matching_is_equally_likely(m, rounds):
    o = matching_fixture(m, 2, seed=5)
    counts = Counter(matchings(o, 2 * t)[0] for t in range(rounds))
    cells = list(permutations(range(m)))
    assert set(counts) <= set(cells)
    assert len(counts) == len(cells)  # every permutation occurs (Sattolo's draws only cycles)
    exp = rounds / len(cells)
    chi2 = sum((counts.get(c, 0) - exp) ** 2 / exp for c in cells)
    assert chi2_sf(chi2, len(cells) - 1) > 1e-6, (chi2, counts)


def test_pairs_and_rounds_draw_independent_matchings():
    """h = 4: pairs (0,1) and (2,3) in even rounds, (1,2) in odd ones.  The two
    pairs of one round agree as often as two independent draws would (1/m!),
    and so do consecutive even rounds of one pair."""
    m, R = 3, 6000
    o = matching_fixture(m, 4, seed=9)
    same_pair, same_round, prev = 0, 0, None
    odd = Counter()
    for t in range(R):
        ev = matchings(o, 2 * t)
        same_pair += ev[0] == ev[2]
        same_round += prev is not None and ev[0] == prev
        prev = ev[0]
        odd[matchings(o, 2 * t + 1)[1]] += 1
    p = 1.0 / math.factorial(m)
    sd = math.sqrt(R * p * (1 - p))
    assert abs(same_pair - R * p) < 5 * sd
    assert abs(same_round - (R - 1) * p) < 5 * sd
    exp = R / 6
    chi2 = sum((odd.get(c, 0) - exp) ** 2 / exp for c in permutations(range(m)))
    assert chi2_sf(chi2, 5) > 1e-6


def test_one_walker_per_window_always_meets_its_neighbour():
    o = matching_fixture(1, 3, seed=2)
    for r in range(6):
        assert all(pi == (0,) for pi in matchings(o, r).values())


def test_matching_from_the_published_shuffle_by_hand():
    """Round 0, windows (0, 1), m = 5, seed 7: Fisher-Yates from the last
    position down, position i swapped with j = floor(w (i + 1) / 2^32), the
    words w taken in order from the Philox blocks (round, n / 4, a, 3)."""
    m, seed = 5, 7
    o = matching_fixture(m, 2, seed)
    key = [seed & 0xffffffff, seed >> 32]
    pi = list(range(m))
    words = list(O.philox4x32_10([0, 0, 0, 3], key)) + list(O.philox4x32_10([0, 1, 0, 3], key))
    for n, i in enumerate(range(m - 1, 0, -1)):
        j = (int(words[n]) * (i + 1)) >> 32
        pi[i], pi[j] = pi[j], pi[i]
    assert matchings(o, 0)[0] == tuple(pi)
