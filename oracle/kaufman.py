"""Exact density of states of the 2D Ising model on the L x L torus.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): the counts pin the REWL
oracle on lattices beyond the reach of enumeration and of the transfer matrix.

Method (Beale, Phys. Rev. Lett. 76, 78 (1996)): Kaufman's exact partition
function of the finite torus (Phys. Rev. 76, 1232 (1949)),

    Z = 1/2 (2 sinh 2K)^(N/2) (Z1 + Z2 + Z3 + Z4),
    Z1 = prod_{k odd} 2 cosh(L g_k / 2),   Z2 = prod_{k odd} 2 sinh(L g_k / 2),
    Z3 = prod_{k even} 2 cosh(L g_k / 2),  Z4 = prod_{k even} 2 sinh(L g_k / 2),
    k = 0 .. 2L - 1,  cosh g_k = cosh 2K coth 2K - cos(pi k / L),
    g_0 = 2K + ln tanh K,

is a polynomial in y = exp(-2K): with b broken bonds (Potts energy
E = b - 2N, Ising energy 2b - 2N), y^N Z = P(y) = sum_b g(b) y^b.  Beale
expands it exactly; here P is evaluated at M points on a circle |y| = rho in
high-precision complex arithmetic and its coefficients are read off by a
discrete Fourier transform, then rounded to integers.

To keep the evaluation free of branch cuts, every factor is written as a
rational function of y: for even L, 2 cosh(L g / 2) = 2 T_{L/2}(cosh g) and
2 sinh(L g / 2) = 2 sinh(g) U_{L/2-1}(cosh g) (Chebyshev polynomials); in the
products the factors of k and 2L - k are equal and pair to
sinh^2 g_k = cosh^2 g_k - 1; the unpaired k = 0 and k = L have
exp(g_0) = (1 - y) / (y (1 + y)) and exp(g_L) = (1 + y) / (y (1 - y)).
"""
import math


def _chebyshev_TU(c, n):
    """(T_n(c), U_{n-1}(c)) by the three-term recurrences."""
    t0, t1 = 1, c
    u0, u1 = 0, 1  # U_{-1}, U_0
    for _ in range(1, n):
        t0, t1 = t1, 2 * c * t1 - t0
        u0, u1 = u1, 2 * c * u1 - u0
    return t1, u1


def _P(y, L, cosk, mp):
    """P(y) = y^N Z(K) at complex y (L even)."""
    N = L * L
    h = L // 2
    y2 = y * y
    A = (1 + y2) ** 2 / (2 * y * (1 - y2))  # cosh 2K coth 2K
    z1 = z2 = z3 = z4 = mp.mpc(1)
    for k in range(2 * L):
        c = A - cosk[k]
        T, U = _chebyshev_TU(c, h)
        if k % 2:
            z1 *= 2 * T
            if k < L:  # pairs (k, 2L - k)
                z2 *= 4 * (c * c - 1) * U * U
        else:
            z3 *= 2 * T
            if 0 < k < L:
                z4 *= 4 * (c * c - 1) * U * U
    X0 = (1 - y) / (y * (1 + y))
    XL = (1 + y) / (y * (1 - y))
    z4 *= (X0 ** h - X0 ** (-h)) * (XL ** h - XL ** (-h))
    pref = ((1 - y2) / y) ** (N // 2)
    return pref * (z1 + z2 + z3 + z4) / 2 * y ** N


def _fft(a, mp, inverse=False):
    """Radix-2 FFT of a list of mpc (length a power of two)."""
    n = len(a)
    if n == 1:
        return list(a)
    even = _fft(a[0::2], mp, inverse)
    odd = _fft(a[1::2], mp, inverse)
    sgn = 1 if inverse else -1
    out = [None] * n
    for k in range(n // 2):
        w = mp.expjpi(sgn * mp.mpf(2 * k) / n) * odd[k]
        out[k] = even[k] + w
        out[k + n // 2] = even[k] - w
    return out


def ising_counts(L, dps=None, rho=0.9):
    """Exact g(b), b = 0 .. 2N broken bonds, of the L x L Ising torus (L even).

    Returns (counts, worst) with the counts as Python integers and worst the
    largest distance of a Fourier coefficient from its integer (a measure of
    the arithmetic's accuracy; well below 0.5 means the rounding is exact)."""
    import mpmath

    if L % 2 or L < 4:
        raise ValueError("L must be even and >= 4")
    N = L * L
    mp = mpmath.mp
    old = mp.dps
    mp.dps = dps or int(0.35 * N + 2.2 * N * math.log10(1 / rho) + 120)
    try:
        rho = mp.mpf(rho)
        cosk = [mp.cospi(mp.mpf(k) / L) for k in range(2 * L)]
        M = 1
        while M < 2 * N + 1:
            M *= 2
        # points rho exp(i pi (2j + 1) / M): none on the real axis, where
        # 1 - y^2 or y would vanish; P has real coefficients, so
        # P(conj y) = conj P(y) and only half the points are evaluated
        vals = [None] * M
        for j in range(M // 2):
            y = rho * mp.expjpi(mp.mpf(2 * j + 1) / M)
            v = _P(y, L, cosk, mp)
            vals[j] = v
            vals[M - 1 - j] = mp.conj(v)
        # sum_j P(y_j) exp(-2 pi i j b / M) = M g(b) rho^b exp(i pi b / M)
        coef = _fft(vals, mp)
        counts, worst = [], mp.mpf(0)
        for b in range(2 * N + 1):
            a = coef[b] * mp.expjpi(-mp.mpf(b) / M) / M / rho ** b
            r = mp.nint(a.real)
            worst = max(worst, abs(a.real - r), abs(a.imag))
            counts.append(int(r))
        return counts, float(worst)
    finally:
        mp.dps = old
