"""Comparison of two REWL runs in which every difference must be traced.

The CUDA path and the oracle take the same decisions on the same Philox draws
(Sec. 2 of arXiv:1312.3004: accept iff D >= 0 or u < exp(D)), except where
|u - exp(D)| is so small that the exp of two libraries can round the
comparison differently.  The CUDA library logs such near ties (walker and step,
or exchange pair and round: REWL_FIELD_TIES); the oracle can invert chosen
decisions.  A difference between the two states is accepted only when
inverting some of the logged near-tie decisions in a fresh oracle run
reproduces the CUDA state exactly -- i.e. the first divergent decision of
every walker involved is a logged near tie -- and each of those decisions was
a near tie for the oracle too.  Anything else fails.
"""
import itertools

import numpy as np

from oracle import oracle as O

INT_FIELDS = ("spins", "energy", "replica", "steps", "hist", "mask", "iter", "done", "trips", "trip_end")
FLOAT_FIELDS = ("lng", "lnf")


def gpu_state(r):
    st = {name: r.get(name) for name in INT_FIELDS}
    for name in FLOAT_FIELDS:
        st[name] = r.get(name).view(np.uint64)
    st["round"] = np.array([r.round])
    return st


def oracle_state(o):
    st = {"spins": o.sigma(), "energy": o.E(), "replica": o.rep(), "steps": o.t(), "hist": o.H(),
          "mask": o.mask(), "iter": o.iter(), "done": o.done(), "trips": o.rt_trips(), "trip_end": o.rt_end(),
          "lng": o.lng().view(np.uint64), "lnf": o.lnf().view(np.uint64), "round": np.array([o.round])}
    return st


def differing(a, b):
    return [k for k in a if not np.array_equal(a[k], b[k])]


def gpu_ties(r):
    """(count, [(kind, who, when), ...]) of the CUDA run's near ties."""
    n = int(r.stats()["near_ties"])
    log = r.get("ties")
    return n, [(int(c >> 32), int(c & 0xffffffff), int(w)) for c, w in log[:min(n, len(log))]]


def planted_near_tie(orc, seed, g, setter=None):
    """Place a near tie at step 0 of walker g of a fresh run: ln g of the first
    proposal's target bin is set so that D = ln g(E) - ln g(E') = ln u, i.e.
    exp(D) = u up to rounding (the proposal and u follow the oracle's reading
    of the WL step).  orc: a fresh oracle run of the instance (it is changed);
    setter(lng): also applies the same ln g to another run.  Returns (D, u), or
    None if the proposal leaves the window or keeps the energy."""
    q, L, m, W = orc.q, orc.L, orc.m, orc.W
    r = O.philox4x32_10([0, 0, g, 0], [seed & 0xffffffff, seed >> 32])
    N = L * L
    site = (int(r[0]) * N) >> 32
    sig = orc.sigma()[g]
    cur = int(sig[site])
    v = (int(r[1]) * (q - 1)) >> 32
    nw = v + (v >= cur)
    x, y = site % L, site // L
    nb = [y * L + (x + 1) % L, y * L + (x - 1) % L, ((y + 1) % L) * L + x, ((y - 1) % L) * L + x]
    dE = sum(int(sig[n] == cur) - int(sig[n] == nw) for n in nb)
    E = int(orc.E()[g])
    lo = int(orc.e_lo()[g // m])
    if dE == 0 or not (lo <= E + dE <= lo + W):
        return None
    u = (((int(r[2]) >> 5) << 26) | (int(r[3]) >> 6)) * 2.0 ** -53
    lng = orc.lng()
    lng[g, E + dE - lo] = -np.log(u)
    orc.set_lng(lng)
    if setter is not None:
        setter(lng)
    return lng[g, E - lo] - lng[g, E + dE - lo], u


class TracedPair:
    """A run of the implementation under test beside oracle runs that follow it.

    make_test(): the run under test (a REWL handle, or anything with run(n),
    and a state / near-tie interface given by state_of / ties_of);
    make_oracle(): a fresh oracle run of the same instance.
    require_oracle_tie: every inverted decision must be a near tie
    (|u - exp(D)| < 2e-14) in the oracle's own arithmetic as well.
    """

    def __init__(self, make_test, make_oracle, state_of=gpu_state, ties_of=gpu_ties, require_oracle_tie=True,
                 max_new=6):
        self.test = make_test()
        self.make_oracle = make_oracle
        self.state_of, self.ties_of = state_of, ties_of
        self.require_oracle_tie = require_oracle_tie
        self.max_new = max_new
        self.inverted = []  # decisions the oracle inverts to follow the run under test
        self.rounds = 0     # rounds asked for so far (None: until converged)
        self.orc = make_oracle()

    def _oracle(self, inverted):
        o = self.make_oracle()
        for d in inverted:
            o.invert_decision(*d)
        if self.rounds is None:
            o.run(0)
        elif self.rounds > 0:
            o.run(self.rounds)
        return o

    def check(self):
        """Assert that the two states agree, or that their difference is traced."""
        got = self.state_of(self.test)
        diff = differing(got, oracle_state(self.orc))
        if not diff:
            return
        n, logged = self.ties_of(self.test)
        assert n > 0, "state differs in %s without a near-tie acceptance draw" % diff
        assert n <= 32, "state differs in %s after %d near ties, more than the log holds" % (diff, n)
        new = [d for d in logged if d not in self.inverted]
        assert new, "state differs in %s; every logged near tie %s is already followed" % (diff, logged)
        assert len(new) <= self.max_new, "too many new near ties to try: %s" % new
        for k in range(1, len(new) + 1):
            for combo in itertools.combinations(new, k):
                o = self._oracle(self.inverted + list(combo))
                if differing(got, oracle_state(o)):
                    continue
                if self.require_oracle_tie:
                    _, seen = o.ties()
                    gaps = {(a, b, c): g for a, b, c, g in seen}
                    for d in combo:
                        assert d in gaps and gaps[d] < 2e-14, (
                            "decision %s explains the difference but is no near tie for the oracle (%s)"
                            % (d, gaps.get(d)))
                self.inverted += list(combo)
                self.orc = o
                return
        raise AssertionError("state differs in %s; no choice of the logged near-tie decisions %s, inverted "
                             "in the oracle, reproduces it" % (diff, new))

    def run(self, n):
        """n rounds of both (n <= 0: until converged), then check()."""
        self.test.run(n)
        self.orc.run(n)
        if n <= 0 or self.rounds is None:
            self.rounds = None
        else:
            self.rounds += n
        self.check()
