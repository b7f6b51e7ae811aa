"""Pins of the exact density-of-states generators (oracle/exact_dos.c).

The generators are checked against each other (brute force vs transfer matrix,
with and without the colour-permutation reduction), against closed-form counts
derived by hand, against the total q^N, and -- for the Ising case q=2 --
against Kaufman's exact partition function of the finite torus evaluated in
high precision, which shares nothing with the transfer-matrix code.  Beyond
the transfer matrix's reach (L = 16, 32) the Ising counts come from Kaufman's
function expanded as a polynomial (Beale's method, oracle/kaufman.py), checked
against the transfer matrix where both run, against low-energy counts derived
by hand, and used to pin the whole oracle on the 16 x 16 torus.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O


@pytest.mark.parametrize("q,L", [(2, 3), (2, 4), (3, 3), (4, 3)])
def test_transfer_matrix_equals_brute_force(q, L):
    bf = O.exact_counts_brute(q, L)
    assert O.exact_counts_tm(q, L, symmetry=False) == bf
    assert O.exact_counts_tm(q, L, symmetry=True) == bf


@pytest.mark.parametrize("q,L", [(3, 4), (2, 5), (4, 4)])
def test_colour_symmetry_reduction(q, L):
    assert O.exact_counts_tm(q, L, symmetry=True) == O.exact_counts_tm(q, L, symmetry=False)


@pytest.mark.parametrize("q,L", [(2, 4), (2, 5), (2, 6), (2, 8), (3, 4), (3, 5), (10, 4)])
def test_total_and_low_energy_closed_forms(q, L):
    """sum g = q^N; with k broken bonds: g(0) = q (uniform states); k = 1, 2, 3, 5
    impossible; k = 4 one odd spin: q(q-1)N; k = 6 an adjacent equal pair:
    2N q(q-1); k = 7 an adjacent pair of two different odd values:
    2N q(q-1)(q-2).  (Valid for L >= 4, where no loop wraps the torus.)"""
    N = L * L
    g = O.exact_counts_tm(q, L)
    assert sum(g) == q ** N
    assert g[0] == q
    for k in (1, 2, 3, 5):
        assert g[k] == 0
    assert g[4] == q * (q - 1) * N
    assert g[6] == 2 * N * q * (q - 1)
    assert g[7] == 2 * N * q * (q - 1) * (q - 2)


@pytest.mark.parametrize("L", [4, 6, 8])
def test_ising_bipartite_symmetry(L):
    """q=2, even L: flipping one sublattice maps k broken bonds to 2N-k; odd k
    never occurs (every single flip changes k by an even amount)."""
    N = L * L
    g = O.exact_counts_tm(2, L)
    for k in range(2 * N + 1):
        assert g[k] == g[2 * N - k]
        if k % 2:
            assert g[k] == 0


def _kaufman_Z(K, L, mp):
    """Kaufman (1949) partition function of the L x L Ising torus,
    Z = 1/2 (2 sinh 2K)^{N/2} (Z1 + Z2 + Z3 + Z4), with
    cosh g_k = cosh 2K coth 2K - cos(pi k / L) and g_0 = 2K + ln tanh K."""
    K = mp.mpf(K)

    def gam(k):
        if k == 0:
            return 2 * K + mp.log(mp.tanh(K))
        return mp.acosh(mp.cosh(2 * K) ** 2 / mp.sinh(2 * K) - mp.cos(mp.pi * k / L))

    z1 = z2 = z3 = z4 = mp.mpf(1)
    for r in range(L):
        g_odd, g_even = gam(2 * r + 1), gam(2 * r)
        z1 *= 2 * mp.cosh(L * g_odd / 2)
        z2 *= 2 * mp.sinh(L * g_odd / 2)
        z3 *= 2 * mp.cosh(L * g_even / 2)
        z4 *= 2 * mp.sinh(L * g_even / 2)
    return (2 * mp.sinh(2 * K)) ** (mp.mpf(L * L) / 2) * (z1 + z2 + z3 + z4) / 2


@pytest.mark.parametrize("L", [4, 8])
def test_ising_counts_match_kaufman(L):
    """Ising energy H = -sum s_i s_j = 2E + 2N for the q=2 Potts energy E, so
    Z(K) = sum_k g(k) exp(-K (2k - 2N)) must equal Kaufman's closed form."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    N = L * L
    g = O.exact_counts_tm(2, L)
    for K in (0.1, 0.3, 0.44068679, 0.6, 1.0):
        z_tm = sum(mp.mpf(c) * mp.exp(-mp.mpf(K) * (2 * k - 2 * N)) for k, c in enumerate(g))
        assert abs(z_tm / _kaufman_Z(K, L, mp) - 1) < mp.mpf(10) ** -40


def test_q10_exact_transition_temperature_constant():
    """The exact q=10 transition temperature quoted in Sec. 3.1 (0.701232) is
    1 / ln(1 + sqrt(q)) (self-duality); checks the constant the tests use."""
    assert abs(1.0 / math.log(1.0 + math.sqrt(10.0)) - 0.701232) < 5e-7


# --------------------------------------------------------------------------
# Beale's exact Ising density of states on larger tori (oracle/kaufman.py):
# Kaufman's torus partition function expanded in y = exp(-2K).
@pytest.mark.parametrize("L", [4, 6, 8])
def test_kaufman_expansion_equals_the_transfer_matrix(L):
    pytest.importorskip("mpmath")
    from oracle import kaufman

    counts, worst = kaufman.ising_counts(L)
    assert worst < 1e-6
    assert counts == O.exact_counts_tm(2, L)


def _stored_exact():
    import json
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "ising_exact_torus.json")
    with open(path) as f:
        return json.load(f)["lattices"]


@pytest.mark.parametrize("L", [16, 32])
def test_stored_exact_ising_counts_obey_closed_forms(L):
    """The stored L = 16 and 32 counts (tests/golden/make_ising_exact.py):
    exact integer rounding (residual far below 1/2); the low-energy counts
    derived by hand for a torus without wrapping clusters, b broken bonds,
    g(b) = 2 x (sets S of flipped spins with 4|S| - 2 adj(S) = b):
    g(0) = 2; g(4) = 2N (one spin); g(6) = 4N (a domino); g(8) = N(N - 1) + 10N
    (two spins not adjacent, straight and bent trominoes, the 2x2 square);
    g(10) = 4N^2 + 24N (a domino and a spin not touching it, the 18 fixed
    tetrominoes other than the square, the 8 P-pentominoes, the 2x3
    rectangles); odd b and b = 2 impossible; sum g = 2^N; and g(b) = g(2N - b)."""
    d = _stored_exact()[str(L)]
    N = L * L
    assert d["N"] == N and d["max_rounding_residual"] < 1e-6
    low = [int(x) for x in d["low_counts"]]
    assert low[:11] == [2, 0, 0, 0, 2 * N, 0, 4 * N, 0, N * (N - 1) + 10 * N, 0, 4 * N * N + 24 * N]
    assert all(low[b] == 0 for b in range(1, 17, 2))
    lng = d["lng"]
    assert len(lng) == 2 * N + 1
    for b in range(2 * N + 1):
        assert (lng[b] is None) == (b % 2 == 1 or b in (2, 2 * N - 2))
        assert lng[b] == lng[2 * N - b]
    v = np.array([x for x in lng if x is not None])
    top = v.max()
    assert abs(top + math.log(np.exp(v - top).sum()) - N * math.log(2.0)) < 1e-12 * N


@pytest.mark.parametrize("L", [16, 32])
def test_stored_exact_ising_counts_give_kaufmans_partition_function(L):
    """sum_b g(b) exp(-K (2b - 2N)) from the stored ln g equals Kaufman's
    closed form evaluated in its usual real form (acosh of cosh g_k, signed
    g_0) at temperatures on both sides of the transition."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    d = _stored_exact()[str(L)]
    N = L * L
    for K in (0.2, 0.4, 0.44068679, 0.5, 0.8):
        terms = [mp.mpf(x) - mp.mpf(K) * (2 * b - 2 * N) for b, x in enumerate(d["lng"]) if x is not None]
        top = max(terms)
        ln_z = top + mp.log(sum(mp.exp(t - top) for t in terms))
        assert abs(ln_z - mp.log(_kaufman_Z(K, L, mp))) < 1e-12 * N


def _l16_run(seed):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from oracle import oracle as OO

    o = OO.OracleREWL(2, 16, 4, 0.75, 2, 1e-6, 0.8, 10_000, seed)
    assert o.run(0)
    return o.lng_joined()


def test_oracle_rewl_reproduces_the_exact_L16_ising_density_of_states():
    """The whole oracle on the 16 x 16 Ising torus (4 windows, 75 % overlap,
    2 walkers each, ln f_final = 1e-6): the visited energies are exactly the
    exact support, and each run's normalised ln g is within the single-run
    bound 0.35 of Beale's exact values (rms below 0.1)."""
    import multiprocessing as mpr

    d = _stored_exact()["16"]
    ex = np.array([x if x is not None else -np.inf for x in d["lng"]])
    fin = np.isfinite(ex)
    with mpr.get_context("spawn").Pool(2) as pool:
        runs = pool.map(_l16_run, [1, 2])
    for lg in runs:
        assert np.array_equal(np.isfinite(lg), fin)
        err = lg[fin] - ex[fin]
        assert np.abs(err).max() < 0.35
        assert np.sqrt((err ** 2).mean()) < 0.1
