"""Pins of the oracle's canonical analysis (oracle/thermo.py).

canonical() is checked against sums over every configuration of small tori
(energies counted here with numpy, not from a density of states), against
Kaufman's closed-form partition function of the Ising torus differentiated in
high precision, against the identity c = du/dT and the T -> 0 / T -> infinity
limits.  equal_peak_temperature() is checked against a two-level closed form,
against brute force over every pair of bins on small inputs, and against its
transformation laws.  bootstrap() is checked against exact pieces with
arbitrary per-window offsets (the join must undo them) and by hand.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from oracle import thermo as TH


def _all_energies(q, L):
    """Potts energy E = -sum over the 2N bonds of delta(s_i, s_j) of every
    configuration of the periodic L x L lattice."""
    N = L * L
    codes = np.arange(q ** N, dtype=np.int64)
    s = np.empty((q ** N, L, L), dtype=np.int8)
    for k in range(N):
        s[:, k // L, k % L] = codes % q
        codes //= q
    sat = (s == np.roll(s, 1, axis=1)).sum(axis=(1, 2)) + (s == np.roll(s, 1, axis=2)).sum(axis=(1, 2))
    return -sat.astype(np.float64)


@pytest.mark.parametrize("q,L", [(3, 3), (2, 4)])
def test_canonical_equals_sums_over_configurations(q, L):
    N = L * L
    E = _all_energies(q, L)
    lng = O.exact_lng(O.exact_counts_brute(q, L))
    Ts = np.array([0.3, 0.7, 1.0, 1.5, 4.0])
    u, c, f, s = TH.canonical(lng, Ts)
    for i, T in enumerate(Ts):
        w = np.exp(-(E - E.min()) / T)
        Z = w.sum()
        e1 = (w * E).sum() / Z
        var = (w * (E - e1) ** 2).sum() / Z
        lnZ = math.log(Z) - E.min() / T
        assert u[i] == pytest.approx(e1 / N, rel=1e-12)
        assert c[i] == pytest.approx(var / (N * T * T), rel=1e-10)
        assert f[i] == pytest.approx(-T * lnZ / N, rel=1e-12)
        assert s[i] == pytest.approx((e1 / N + T * lnZ / N) / T, rel=1e-11)


def test_canonical_matches_kaufman_ising_torus():
    """q = 2, L = 8: ln Z_Potts(beta) = N beta + ln Z_Ising(K = beta / 2) (the
    Ising energy is 2E + 2N); u = -d ln Z / d beta / N and
    c = beta^2 d^2 ln Z / d beta^2 / N, differentiated with mpmath."""
    mp = pytest.importorskip("mpmath")
    from test_oracle_exact import _kaufman_Z
    mp.mp.dps = 50
    L, N = 8, 64
    lng = O.exact_lng(O.exact_counts_tm(2, L))

    def lnZ(beta):
        return N * beta + mp.log(_kaufman_Z(beta / 2, L, mp))

    for T in (0.8, 1.1346, 1.3, 2.5):
        beta = mp.mpf(1) / T
        u_ex = -mp.diff(lnZ, beta) / N
        c_ex = beta ** 2 * mp.diff(lnZ, beta, 2) / N
        f_ex = -lnZ(beta) / beta / N
        u, c, f, s = TH.canonical(lng, [T])
        assert u[0] == pytest.approx(float(u_ex), rel=1e-12)
        assert c[0] == pytest.approx(float(c_ex), rel=1e-10)
        assert f[0] == pytest.approx(float(f_ex), rel=1e-12)
        assert s[0] == pytest.approx(float((u_ex - f_ex) * beta), rel=1e-11)


def test_specific_heat_is_the_temperature_derivative_of_u():
    lng = O.exact_lng(O.exact_counts_tm(3, 4))
    for T in (0.5, 0.9, 1.4):
        d = 1e-5
        u = TH.canonical(lng, [T - d, T + d])[0]
        assert TH.canonical(lng, [T])[1][0] == pytest.approx((u[1] - u[0]) / (2 * d), rel=1e-6)


@pytest.mark.parametrize("q,L", [(2, 4), (3, 4), (10, 4)])
def test_high_and_low_temperature_limits(q, L):
    """T -> infinity: every bond satisfied with probability 1/q, so u -> -2/q,
    s -> ln q; T -> 0: the q ground states, u -> -2, s -> ln(q) / N."""
    N = L * L
    lng = O.exact_lng(O.exact_counts_tm(q, L))
    u, c, f, s = TH.canonical(lng, [1e7])
    assert u[0] == pytest.approx(-2.0 / q, abs=1e-5)
    assert s[0] == pytest.approx(math.log(q), abs=1e-6)
    u, c, f, s = TH.canonical(lng, [0.02])
    assert u[0] == pytest.approx(-2.0, abs=1e-12)
    assert s[0] == pytest.approx(math.log(q) / N, abs=1e-12)
    assert c[0] == pytest.approx(0.0, abs=1e-12)


def test_specific_heat_peak_matches_a_fine_scan_over_configurations():
    q, L = 3, 3
    N = L * L
    E = _all_energies(q, L)
    Ts = np.linspace(0.4, 1.6, 24001)
    best = (-1.0, 0.0)
    for T in Ts:
        w = np.exp(-(E - E.min()) / T)
        e1 = (w * E).sum() / w.sum()
        c = (w * (E - e1) ** 2).sum() / w.sum() / (N * T * T)
        best = max(best, (c, T))
    T_pk, c_pk = TH.specific_heat_peak(O.exact_lng(O.exact_counts_brute(q, L)), 0.4, 1.6)
    assert T_pk == pytest.approx(best[1], abs=1e-4)
    assert c_pk == pytest.approx(best[0], rel=1e-8)
    assert c_pk >= best[0] * (1 - 1e-12)


def test_canonical_distribution_scaled_to_one():
    lng = O.exact_lng(O.exact_counts_tm(3, 4))
    p = TH.canonical_distribution(lng, 0.8)
    assert p.max() == 1.0
    assert np.all(p[~np.isfinite(lng)] == 0)
    N, E = 16, np.arange(33) - 32
    ok = np.isfinite(lng)
    ratio = p[ok] / np.exp(lng[ok] - E[ok] / 0.8)
    assert np.allclose(ratio, ratio[0], rtol=1e-12)


def test_two_level_equal_peak_closed_form():
    """Only two energies: the peaks are equal where ln g1 - E1/T = ln g2 - E2/T."""
    lng = np.full(17, -np.inf)
    lng[2], lng[12] = 1.0, 9.5
    T, e_lo, e_hi, ln_sup = TH.equal_peak_temperature(lng, 0.1, 10.0)
    assert T == pytest.approx(10.0 / 8.5, rel=1e-15)
    assert (e_lo, e_hi) == (2 - 16, 12 - 16)
    assert ln_sup == 0.0
    assert TH.equal_peak_temperature(lng, 2.0, 10.0) is None
    # A third energy just under the line between the two is a transition state
    # (suppressed by 1e-7 in ln P), just above it a peak of its own.
    chord = 1.0 + (9.5 - 1.0) * (7 - 2) / 10
    lng[7] = chord - 1e-7
    T, e_lo, e_hi, ln_sup = TH.equal_peak_temperature(lng, 0.1, 10.0)
    assert (e_lo, e_hi) == (-14, -4)
    assert ln_sup == pytest.approx(-1e-7, rel=1e-6)
    lng[7] = chord + 1e-7
    T, e_lo, e_hi, ln_sup = TH.equal_peak_temperature(lng, 0.1, 10.0)
    assert e_hi - e_lo == 5 and ln_sup == 0.0


def _intruder(nb, rng, depth=3.0):
    """A concave ln g with a convex dent (a first-order signature) and noise."""
    x = np.linspace(-1, 1, nb)
    lg = 40 * (1 - x * x) + 0.6 * 40 * x
    lg -= depth * np.exp(-((x + 0.05) / 0.2) ** 2)
    return lg + 0.01 * rng.standard_normal(nb)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_equal_peak_brute_force_over_pairs(seed):
    """Every pair (i, j) whose bins are both global maxima of ln g - E/T at the
    pair's own slope is an equal-peak pair; the widest one with T in range is
    the double peak."""
    rng = np.random.default_rng(seed)
    nb = 41
    lng = _intruder(nb, rng)
    lng[rng.choice(nb, 4, replace=False)] = -np.inf
    N, E = (nb - 1) // 2, np.arange(nb) - (nb - 1)
    T_lo, T_hi = 0.05, 50.0
    best = None
    fin = np.flatnonzero(np.isfinite(lng))
    for i, j in itertools.combinations(fin, 2):
        beta = (lng[j] - lng[i]) / (E[j] - E[i])
        if beta <= 0 or not (T_lo <= 1 / beta <= T_hi):
            continue
        a = lng[fin] - E[fin] * beta
        top = max(lng[i] - E[i] * beta, lng[j] - E[j] * beta)
        if a.max() > top + 1e-9:
            continue
        if best is None or E[j] - E[i] > best[0]:
            best = (E[j] - E[i], 1 / beta, E[i], E[j])
    T, e_lo, e_hi, ln_sup = TH.equal_peak_temperature(lng, T_lo, T_hi)
    assert (e_lo, e_hi) == (best[2], best[3])
    assert T == pytest.approx(best[1], rel=1e-12)
    p = TH.canonical_distribution(lng, T)
    assert p[e_lo + 2 * N] == pytest.approx(1.0, abs=1e-9)
    assert p[e_hi + 2 * N] == pytest.approx(1.0, abs=1e-9)
    inner = p[e_lo + 2 * N:e_hi + 2 * N + 1]
    assert math.log(inner[inner > 0].min()) == pytest.approx(ln_sup, abs=1e-9)
    assert ln_sup < 0


def test_equal_peak_transformation_laws():
    """ln g + C leaves Tc unchanged; ln g + kE shifts 1/Tc by k."""
    lng = _intruder(61, np.random.default_rng(7))
    T0, a0, b0, s0 = TH.equal_peak_temperature(lng, 0.05, 50.0)
    T1, a1, b1, s1 = TH.equal_peak_temperature(lng + 123.25, 0.05, 50.0)
    assert (T1, a1, b1) == (pytest.approx(T0, rel=1e-13), a0, b0)
    E = np.arange(61) - 60
    T2, a2, b2, s2 = TH.equal_peak_temperature(lng + 0.125 * E, 0.05, 50.0)
    assert (a2, b2) == (a0, b0)
    assert 1 / T2 == pytest.approx(1 / T0 + 0.125, rel=1e-12)
    assert s2 == pytest.approx(s0, abs=1e-10)


def _exact_pieces(q, L, h, overlap, rng, offsets=True):
    N = L * L
    lng = O.exact_lng(O.exact_counts_tm(q, L))
    e_lo, W = O.window_table(L, h, overlap)
    lw = np.zeros((h, W + 1))
    mw = np.zeros((h, W + 1), dtype=np.uint8)
    for a in range(h):
        seg = lng[e_lo[a] + 2 * N:e_lo[a] + 2 * N + W + 1]
        mw[a] = np.isfinite(seg)
        lw[a] = np.where(mw[a] != 0, seg, 0.0) + (rng.uniform(-50, 50) if offsets else 0.0)
    return lng, e_lo, W, lw, mw


def test_bootstrap_of_offset_exact_pieces_is_exact():
    """Pieces that are the exact ln g plus an arbitrary constant per run and
    window: whatever runs a resample draws, the join removes the constants."""
    q, L, h, o = 3, 5, 4, 0.75
    N = L * L
    rng = np.random.default_rng(11)
    runs = [_exact_pieces(q, L, h, o, rng) for _ in range(5)]
    lng, e_lo, W = runs[0][0], runs[0][1], runs[0][2]
    lw = np.stack([r[3] for r in runs])
    mw = np.stack([r[4] for r in runs])
    draws = rng.integers(0, 5, size=(6, 5))
    out = TH.bootstrap(q, N, e_lo, W, lw, mw, draws)
    ref = lng - (np.logaddexp.reduce(lng[np.isfinite(lng)]) - N * math.log(q))
    for row in out:
        assert np.array_equal(np.isfinite(row), np.isfinite(lng))
        assert np.allclose(row[np.isfinite(lng)], ref[np.isfinite(lng)], atol=1e-9)


def test_bootstrap_averages_by_hand():
    lw = np.array([[[1.0, 2.0, 3.0]], [[5.0, 0.0, 7.0]]])
    mw = np.array([[[1, 1, 0]], [[1, 0, 1]]], dtype=np.uint8)
    mean, mask = TH.average_pieces(lw, mw, [0, 1])
    assert mean.tolist() == [[3.0, 2.0, 7.0]]
    assert mask.tolist() == [[1, 1, 1]]
    mean, mask = TH.average_pieces(lw, mw, [0, 0])
    assert mean.tolist() == [[1.0, 2.0, 0.0]] and mask.tolist() == [[1, 1, 0]]


def test_bootstrap_of_single_runs_is_their_own_joined_result():
    runs = []
    for seed in (3, 4):
        o = O.OracleREWL(3, 4, 3, 0.75, 2, 1e-3, 0.8, 500, seed)
        assert o.run(0)
        runs.append(o)
    h, W, N = 3, runs[0].W, runs[0].N
    lw = np.stack([r.lng()[::2] for r in runs])     # walker 0 of each window (m = 2)
    mw = np.stack([r.mask() for r in runs])
    out = TH.bootstrap(3, N, runs[0].e_lo(), W, lw, mw, [[0, 0], [1, 1], [1, 0]])
    assert np.array_equal(out[0], runs[0].lng_joined())
    assert np.array_equal(out[1], runs[1].lng_joined())
    assert not np.array_equal(out[2], out[0])
