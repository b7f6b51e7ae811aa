"""The library's analysis calls (host code behind include/rewl.h) against the
oracle's canonical analysis (oracle/thermo.py, pinned in test_oracle_thermo.py).

These functions do no device work, so they run here on the CPU: on exact
densities of states, on densities of states the oracle's REWL produced (noisy,
as real runs are), and on synthetic first-order shapes.
"""
import math

import numpy as np
import pytest

import paper_1312_3004_gb300 as P
from oracle import oracle as O
from oracle import thermo as TH

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _lib_or_skip():
    try:
        P.load()
    except Exception as e:  # the CUDA library is built by build(); nvcc is required
        pytest.skip("librewl.so not built: %s" % e)


@pytest.fixture(scope="module")
def converged_runs():
    runs = []
    for seed in (5, 6, 7):
        o = O.OracleREWL(10, 6, 4, 0.75, 2, 1e-4, 0.8, 2000, seed)
        assert o.run(0)
        runs.append(o)
    return runs


def _cases(converged_runs):
    out = [("exact q2 L8", O.exact_lng(O.exact_counts_tm(2, 8))),
           ("exact q3 L5", O.exact_lng(O.exact_counts_tm(3, 5))),
           ("exact q10 L4", O.exact_lng(O.exact_counts_tm(10, 4)))]
    for k, o in enumerate(converged_runs):
        out.append(("oracle q10 L6 run %d" % k, o.lng_joined()))
    return out


def test_canonical_matches_oracle(converged_runs):
    _lib_or_skip()
    Ts = np.array([0.3, 0.55, 0.70, 0.71, 0.9, 1.2, 3.0, 50.0])
    for name, lng in _cases(converged_runs):
        got = P.canonical(lng, Ts)
        ref = TH.canonical(lng, Ts)
        N = (len(lng) - 1) // 2
        for k, (g, r) in enumerate(zip(got, ref)):
            if k == 1:
                # The oracle forms <E^2> - <E>^2 as written, which loses
                # eps <E^2> / (N T^2) = eps (c + u^2 N / T^2) to cancellation;
                # the library subtracts the mean first.
                tol = 1e-13 * (ref[1] + ref[0] ** 2 * N / Ts ** 2) + 1e-11 * ref[1]
                assert np.all(np.abs(g - r) <= tol), name
            else:
                assert np.allclose(g, r, rtol=1e-12, atol=1e-14), name


def test_canonical_distribution_matches_oracle(converged_runs):
    _lib_or_skip()
    for name, lng in _cases(converged_runs):
        for T in (0.6, 0.7012, 1.5):
            assert np.allclose(P.canonical_distribution(lng, T), TH.canonical_distribution(lng, T),
                               rtol=1e-13, atol=1e-300), name


def test_specific_heat_peak_matches_oracle(converged_runs):
    _lib_or_skip()
    for name, lng in _cases(converged_runs):
        T, c = P.specific_heat_peak(lng, 0.4, 2.0)
        T_ref, c_ref = TH.specific_heat_peak(lng, 0.4, 2.0)
        assert T == pytest.approx(T_ref, rel=1e-6), name
        assert c == pytest.approx(c_ref, rel=1e-10), name


def test_equal_peak_temperature_matches_oracle(converged_runs):
    _lib_or_skip()
    rng = np.random.default_rng(3)
    x = np.linspace(-1, 1, 201)
    synthetic = 80 * (1 - x * x) + 48 * x - 6 * np.exp(-((x + 0.05) / 0.2) ** 2) + 0.02 * rng.standard_normal(201)
    cases = _cases(converged_runs) + [("synthetic", synthetic)]
    for name, lng in cases:
        for lo, hi in ((0.05, 50.0), (0.6, 0.8)):
            ref = TH.equal_peak_temperature(lng, lo, hi)
            if ref is None:
                with pytest.raises(P.RewlError):
                    P.equal_peak_temperature(lng, lo, hi)
                continue
            T, a, b, s = P.equal_peak_temperature(lng, lo, hi)
            assert (a, b) == (ref[1], ref[2]), name
            assert T == pytest.approx(ref[0], rel=1e-14), name
            assert s == pytest.approx(ref[3], rel=1e-12, abs=1e-12), name


def test_two_level_closed_form_through_the_library():
    _lib_or_skip()
    lng = np.full(17, -np.inf)
    lng[2], lng[12] = 1.0, 9.5
    T, a, b, s = P.equal_peak_temperature(lng, 0.1, 10.0)
    assert T == 10.0 / 8.5 and (a, b, s) == (-14, -4, 0.0)
    with pytest.raises(P.RewlError):
        P.equal_peak_temperature(lng, 2.0, 10.0)


def test_join_matches_oracle(converged_runs):
    _lib_or_skip()
    for o in converged_runs:
        e_lo, W = o.e_lo(), o.W
        lw, mw = o.lng()[::o.m], o.mask()
        got = P.join(o.q, o.L, e_lo, W, lw, mw)
        assert np.array_equal(got, o.lng_joined())


def test_bootstrap_matches_oracle(converged_runs):
    _lib_or_skip()
    o0 = converged_runs[0]
    lw = np.stack([o.lng()[::o.m] for o in converged_runs])
    mw = np.stack([o.mask() for o in converged_runs])
    draws = np.random.default_rng(9).integers(0, 3, size=(8, 3))
    got = P.bootstrap(o0.q, o0.L, o0.e_lo(), o0.W, lw, mw, draws)
    ref = TH.bootstrap(o0.q, o0.N, o0.e_lo(), o0.W, lw, mw, draws)
    assert got.shape == ref.shape
    assert np.array_equal(np.isfinite(got), np.isfinite(ref))
    assert np.allclose(got[np.isfinite(got)], ref[np.isfinite(ref)], rtol=0, atol=1e-12)


def test_bootstrap_of_offset_exact_pieces_is_exact():
    """Whatever runs a resample draws, per-run, per-window constants vanish."""
    _lib_or_skip()
    q, L, h, o = 3, 5, 4, 0.75
    N = L * L
    lng = O.exact_lng(O.exact_counts_tm(q, L))
    e_lo, W = O.window_table(L, h, o)
    rng = np.random.default_rng(4)
    lw = np.zeros((4, h, W + 1))
    mw = np.zeros((4, h, W + 1), dtype=np.uint8)
    for r in range(4):
        for a in range(h):
            seg = lng[e_lo[a] + 2 * N:e_lo[a] + 2 * N + W + 1]
            mw[r, a] = np.isfinite(seg)
            lw[r, a] = np.where(mw[r, a] != 0, seg, 0.0) + rng.uniform(-30, 30)
    out = P.bootstrap(q, L, e_lo, W, lw, mw, rng.integers(0, 4, size=(5, 4)))
    ref = lng - (np.logaddexp.reduce(lng[np.isfinite(lng)]) - N * math.log(q))
    for row in out:
        assert np.allclose(row[np.isfinite(lng)], ref[np.isfinite(lng)], atol=1e-9)
        assert not np.isfinite(row[~np.isfinite(lng)]).any()


def test_analysis_arguments_are_checked():
    _lib_or_skip()
    good = O.exact_lng(O.exact_counts_tm(2, 4))
    with pytest.raises(P.RewlError):
        P.canonical(good[:-1], [1.0])                 # even length
    with pytest.raises(P.RewlError):
        P.canonical(np.full(33, -np.inf), [1.0])      # no finite bin
    bad = good.copy()
    bad[3] = np.nan
    with pytest.raises(P.RewlError):
        P.canonical(bad, [1.0])
    for T in (0.0, -1.0, np.inf, np.nan):
        with pytest.raises(P.RewlError):
            P.canonical(good, [T])
        with pytest.raises(P.RewlError):
            P.canonical_distribution(good, T)
    with pytest.raises(P.RewlError):
        P.specific_heat_peak(good, 1.0, 1.0)
    e_lo, W = O.window_table(4, 2, 0.75)
    lw = np.zeros((2, W + 1))
    mw = np.ones((2, W + 1), dtype=np.uint8)
    with pytest.raises(P.RewlError):
        P.join(2, 4, e_lo[::-1], W, lw, mw)           # decreasing window table
    with pytest.raises(P.RewlError):
        P.bootstrap(2, 4, e_lo, W, lw[None], mw[None], [[1]])  # draw outside [0, runs)
    assert P.canonical(good, []) [0].size == 0


def test_ising_energy_equals_the_spin_sum_on_every_configuration():
    """rewl_ising_energy(L, b) against E_I = -sum over bonds of s_i s_j with
    s = +-1, summed directly over every configuration of the 3x3 and 4x4 tori."""
    _lib_or_skip()
    for L in (3, 4):
        N = L * L
        codes = np.arange(2 ** N, dtype=np.int64)
        s = ((codes[:, None] >> np.arange(N)) & 1).reshape(-1, L, L).astype(np.int64) * 2 - 1
        e_ising = -(s * np.roll(s, 1, axis=1)).sum(axis=(1, 2)) - (s * np.roll(s, 1, axis=2)).sum(axis=(1, 2))
        broken = (s != np.roll(s, 1, axis=1)).sum(axis=(1, 2)) + (s != np.roll(s, 1, axis=2)).sum(axis=(1, 2))
        table = {b: P.ising_energy(L, b) for b in range(2 * N + 1)}
        assert all(table[int(b)] == int(e) for b, e in zip(broken, e_ising))
    assert (P.ising_energy(8, 0), P.ising_energy(8, 128), P.ising_energy(8, 4)) == (-128, 128, -120)
    for bad in ((8, -1), (8, 129), (2, 0)):
        with pytest.raises(P.RewlError):
            P.ising_energy(*bad)


def test_join_without_a_common_bin_is_a_state_error():
    """Two windows whose visited bins do not overlap cannot be joined (Fig. 2
    needs a bin where both slopes exist): the library and the oracle refuse."""
    _lib_or_skip()
    e_lo, W = O.window_table(4, 2, 0.75)
    lw = np.zeros((2, W + 1))
    mw = np.zeros((2, W + 1), dtype=np.uint8)
    mw[0, :3] = 1      # the lower window visited only its first bins
    mw[1, -3:] = 1     # the upper window only its last ones
    with pytest.raises(P.RewlError) as err:
        P.join(2, 4, e_lo, W, lw, mw)
    assert err.value.status == 6
    with pytest.raises(RuntimeError):
        O.join_pieces(16, e_lo, W, lw, mw)
