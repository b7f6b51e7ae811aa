"""Pins of the exact density-of-states generators (oracle/exact_dos.c).

The generators are checked against each other (brute force vs transfer matrix,
with and without the colour-permutation reduction), against closed-form counts
derived by hand, against the total q^N, and -- for the Ising case q=2 --
against Kaufman's exact partition function of the finite torus evaluated in
high precision, which shares nothing with the transfer-matrix code.
"""
import math

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
