"""The divergence tracer of the parity tests, checked on the CPU.

A planted difference is made in the oracle only: one oracle run inverts a
chosen acceptance decision (Sec. 2's min[1, g(E)/g(E')], or Eq. 1 for an
exchange) and stands in for the implementation under test.  The tracer must
follow it when the decision is in the near-tie log it is given, and fail when
the log is empty or names another decision.  The oracle's own near-tie log is
pinned by a draw placed within 1e-16 of exp(D).
"""
import numpy as np
import pytest

from oracle import oracle as O
from tie_trace import TracedPair, differing, oracle_state, planted_near_tie

ARGS = (3, 5, 2, 0.75, 2, 1e-3, 0.8, 200, 11)  # q=3, L=5, 2 windows of 2 walkers, K=200


def planted(*decisions):
    def make():
        o = O.OracleREWL(*ARGS)
        for d in decisions:
            o.invert_decision(*d)
        return o
    return make


def fake_log(entries):
    return lambda _o: (len(entries), list(entries))


def test_an_inverted_decision_changes_the_run():
    a, b = planted()(), planted((0, 1, 37))()
    a.run(2)
    b.run(2)
    assert differing(oracle_state(a), oracle_state(b))


def test_identical_runs_pass_without_a_log():
    tp = TracedPair(planted(), planted(), state_of=oracle_state, ties_of=fake_log([]))
    for n in (1, 3):
        tp.run(n)
    assert tp.inverted == []


def test_a_logged_decision_is_followed():
    dec = (0, 1, 37)
    tp = TracedPair(planted(dec), planted(), state_of=oracle_state, ties_of=fake_log([dec]),
                    require_oracle_tie=False)
    tp.run(1)
    tp.run(3)
    assert tp.inverted == [dec]


def test_the_right_decision_is_picked_among_several():
    dec = (0, 2, 150)
    log = [(0, 0, 10), dec, (1, 0, 0)]
    tp = TracedPair(planted(dec), planted(), state_of=oracle_state, ties_of=fake_log(log), require_oracle_tie=False)
    tp.run(4)
    assert tp.inverted == [dec]


def test_an_exchange_decision_is_followed():
    # find an exchange pair that was evaluated in round 0 (windows 0 and 1)
    o = O.OracleREWL(*ARGS)
    o.run(1)
    assert o.xstats()[0] > 0
    for k in range(2):
        dec = (1, k, 0)
        b = planted(dec)()
        b.run(1)
        if differing(oracle_state(o), oracle_state(b)):
            break
    else:
        pytest.skip("no exchange decision of round 0 changes the state")
    tp = TracedPair(planted(dec), planted(), state_of=oracle_state, ties_of=fake_log([dec]),
                    require_oracle_tie=False)
    tp.run(3)
    assert tp.inverted == [dec]


def test_a_difference_without_a_near_tie_fails():
    tp = TracedPair(planted((0, 1, 37)), planted(), state_of=oracle_state, ties_of=fake_log([]))
    with pytest.raises(AssertionError, match="without a near-tie"):
        tp.run(1)


def test_a_difference_at_another_decision_fails():
    tp = TracedPair(planted((0, 1, 37)), planted(), state_of=oracle_state, ties_of=fake_log([(0, 1, 38), (0, 0, 37)]),
                    require_oracle_tie=False)
    with pytest.raises(AssertionError, match="reproduces it"):
        tp.run(1)


def test_a_followed_decision_must_be_a_near_tie_for_the_oracle():
    dec = (0, 1, 37)
    tp = TracedPair(planted(dec), planted(), state_of=oracle_state, ties_of=fake_log([dec]))
    with pytest.raises(AssertionError, match="no near tie for the oracle"):
        tp.run(1)


def test_the_oracle_logs_a_planted_near_tie():
    for g in range(4):
        orc = O.OracleREWL(*ARGS)
        got = planted_near_tie(orc, 11, g)
        if got:
            break
    else:
        pytest.skip("no walker's first proposal stays in its window")
    D, u = got
    assert abs(u - np.exp(D)) < 1e-15
    orc.run(1)
    n, log = orc.ties()
    assert n >= 1
    hit = [e for e in log if e[:3] == (0, g, 0)]
    assert hit and hit[0][3] < 1e-14


def test_decision_counts_of_flat_weights():
    """The counts behind the roofline's exp fraction: with ln g flat and
    ln f = 0 every decision inside the window has D = 0 (none needs exp, every
    one accepts); in an ordinary run some have D < 0, and no count exceeds the
    steps made."""
    o = O.OracleREWL(*ARGS)
    o.production_start(4)  # ln f = 0; ln g is still all zero
    o.production_run(2)
    n, neg = o.decision_counts()
    assert n > 0 and neg == 0
    assert n <= int(o.t().sum())
    r = O.OracleREWL(*ARGS)
    r.run(3)
    n2, neg2 = r.decision_counts()
    assert 0 < neg2 < n2 <= int(r.t().sum())
