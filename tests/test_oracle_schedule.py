"""Pins of the oracle's 1/t ln f schedule (Belardinelli & Pereyra, Phys. Rev. E
75, 046701 (2007); Sec. 2 of arXiv:1312.3004 admits any valid WL update rule).

- Before any window switches to ln f = 1/t, the rule is plain WL with the
  criterion "every bin visited": it must equal the halving schedule run with a
  flatness threshold so small that min H >= p * mean H means min H >= 1.
- After the switch, ln f * (WL steps per walker) = bins in the mask at every
  barrier, and the switch happens at the first halving that would go below 1/t.
- The point of the rule: with halving the error of ln g stalls (about 0.1 on
  these lattices whatever ln f_final), with 1/t it keeps falling as
  ln f_final falls.  Checked against exact densities of states.
"""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _state(o):
    return (o.sigma(), o.E(), o.rep(), o.t(), o.lng(), o.H(), o.mask(), o.lnf(), o.iter(), o.done())


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("q,L,h,m,K,seed", [(3, 4, 3, 2, 700, 1), (10, 5, 2, 3, 1500, 2), (2, 6, 4, 2, 900, 3)])
def test_before_the_switch_the_rule_is_wl_with_every_bin_visited(q, L, h, m, K, seed):
    a = O.OracleREWL(q, L, h, 0.75, m, 1e-6, 0.8, K, seed)
    a.set_schedule(1)
    b = O.OracleREWL(q, L, h, 0.75, m, 1e-6, 1e-12, K, seed)
    rounds = 0
    while not a.phase().any() and rounds < 400:
        assert _same(_state(a), _state(b))
        a.run(1)
        b.run(1)
        rounds += 1
    assert a.iter().sum() > 0          # iterations ended under the "all visited" rule
    assert a.phase().any()             # and the 1/t stage was reached


def test_walker_visited_all_by_hand():
    o = O.OracleREWL(3, 4, 1, 0.75, 2, 1e-3, 0.8, 10, 1)
    B = o.B
    mask = np.zeros((1, B), dtype=np.uint8)
    mask[0, [3, 5, 9]] = 1
    H = np.zeros((2, B), dtype=np.uint32)
    H[0, [3, 5, 9]] = [1, 7, 2]
    H[1, [3, 9, 11]] = [4, 4, 4]          # bin 5 of the mask never visited by walker 1
    o.set_mask(mask)
    o.set_H(H)
    assert o.walker_visited_all(0)
    assert not o.walker_visited_all(1)
    o.set_mask(np.zeros((1, B), dtype=np.uint8))
    assert not o.walker_visited_all(0)   # an empty mask is never "all visited"


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_after_the_switch_lnf_is_one_over_t(seed):
    q, L, h, m, K = 3, 4, 3, 2, 700
    o = O.OracleREWL(q, L, h, 0.75, m, 1e-4, 0.8, K, seed)
    o.set_schedule(1)
    prev_phase = np.zeros(h, dtype=np.uint8)
    prev_lnf = o.lnf()
    switched = 0
    for _ in range(3000):
        if o.done().all():
            break
        o.run(1)
        phase, lnf, t, mask = o.phase(), o.lnf(), o.t(), o.mask()
        for w in range(h):
            n_bins = int(mask[w].sum())
            steps = int(t[w * m])
            if phase[w]:
                assert lnf[w] * steps == pytest.approx(n_bins, rel=1e-15)
                if not prev_phase[w]:    # switched at this barrier: the half went below 1/t
                    assert prev_lnf[w] / 2 < n_bins / steps
                    switched += 1
            else:
                assert lnf[w] in (prev_lnf[w], prev_lnf[w] / 2)
                if lnf[w] != prev_lnf[w]:
                    assert lnf[w] >= n_bins / steps
        prev_phase, prev_lnf = phase, lnf
    assert o.done().all() and switched == h


def _max_error(o, exact):
    lng = o.lng_joined()
    fin = np.isfinite(exact)
    assert np.array_equal(np.isfinite(lng), fin)
    return float(np.max(np.abs(lng[fin] - exact[fin])))


def test_one_over_t_error_keeps_falling_where_halving_stalls():
    q, L, h, m, K = 3, 4, 3, 2, 1000
    N = L * L
    ex = O.exact_lng(O.exact_counts_tm(q, L))
    ex = ex - (np.logaddexp.reduce(ex[np.isfinite(ex)]) - N * np.log(q))
    err = {}
    for sched in (0, 1):
        for lff in (1e-4, 1e-5):
            e = []
            for seed in range(1, 7):
                o = O.OracleREWL(q, L, h, 0.75, m, lff, 0.8, K, seed)
                o.set_schedule(sched)
                assert o.run(20000)
                e.append(_max_error(o, ex))
            err[sched, lff] = np.median(e)
    # halving: no gain from the last decade of ln f_final (saturation)
    assert err[0, 1e-5] > 0.6 * err[0, 1e-4]
    # 1/t: the error keeps falling, by about sqrt(10) per decade, below halving's floor
    assert err[1, 1e-5] < 0.5 * err[1, 1e-4]
    assert err[1, 1e-5] < 0.5 * err[0, 1e-5]
    assert err[1, 1e-5] < 0.06
