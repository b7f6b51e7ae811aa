"""Canonical analysis of a density of states, plain numpy in binary64.

TEST INFRASTRUCTURE ONLY, like the rest of this package: the tests and the
benchmark's reference leg use it to check the library's analysis calls.

Conventions (those of the joined ln g the method produces, Sec. 2 / Fig. 2):
lng[b] = ln g(E) with E = b - 2N for b = 0 .. 2N, -inf where no configuration
exists.  Temperatures in units of J / k_B.

Each function writes its definition out directly:
  canonical            Z(T) = sum_E g(E) exp(-E/T) (the canonical distribution
                       P(E) ~ g(E) exp(-E/T) of Sec. 3.1, Fig. 3b) and the
                       averages taken with it: u = <E>/N, the specific heat
                       c = (<E^2> - <E>^2) / (N T^2), f = -T ln Z / N and
                       s = (u - f) / T.
  canonical_distribution  P(E) scaled to 1 at its highest point (Fig. 3b shows
                       it "normalised to 1 at the peaks").
  specific_heat_peak   the largest c(T) on [T_lo, T_hi]: a grid, then a bounded
                       scalar minimiser (scipy) around the best grid point.
  equal_peak_temperature  Tc(L) as the temperature at which P(E) has two
                       maxima of equal height (Sec. 3.1: the finite-size
                       transition temperature 0.70126 of L = 300, Fig. 3b),
                       from the definition: bin i is a global maximum of
                       ln g(E) - E/T exactly when 1/T lies between the
                       largest slope to a higher bin and the smallest slope
                       from a lower bin; two successive such bins are equal
                       maxima at the slope between them.  Of the pairs whose
                       temperature is in [T_lo, T_hi], the one farthest apart
                       in energy (ties: the lower one) is the double peak.
                       Also returns ln of the suppression of the transition
                       states: min over the energies between the peaks of
                       P(E) / P(peak) (10^-14 at L = 300, Sec. 3.1).
  combine_heo / canonical_observable  the production run's H(E,O) (fixed
                       weights 1/g(E), Sec. 3.2) summed over the windows that
                       cover each energy gives the microcanonical distribution
                       P(O|E) = H(E,O) / sum_O H(E,O); the canonical average is
                       <O>(T) = sum_E g(E) exp(-E/T) <O>_E / sum_E g(E) exp(-E/T)
                       over the energies with finite ln g and production counts.
  bootstrap            error estimate by resampling repeated runs (end of
                       Sec. 2): resample k takes runs draws[k, :], averages
                       their window pieces bin by bin (over the runs that
                       visited the bin), and joins the averages with the
                       oracle's join, so the joining points move from one
                       resample to the next.
"""
import numpy as np

from . import oracle as _orc


def _energies(lng):
    nb = len(lng)
    if nb < 3 or nb % 2 == 0:
        raise ValueError("ln g must have 2N + 1 bins")
    N = (nb - 1) // 2
    return N, np.arange(nb, dtype=np.float64) - 2 * N


def canonical(lng, T):
    """(u, c, f, s) per spin at each temperature of T (arrays of len(T))."""
    lng = np.asarray(lng, dtype=np.float64)
    N, E = _energies(lng)
    ok = np.isfinite(lng)
    lg, E = lng[ok], E[ok]
    T = np.atleast_1d(np.asarray(T, dtype=np.float64))
    u = np.empty(len(T)); c = np.empty(len(T)); f = np.empty(len(T)); s = np.empty(len(T))
    for i, t in enumerate(T):
        a = lg - E / t
        amax = a.max()
        w = np.exp(a - amax)          # g(E) exp(-E/T) / exp(amax)
        Z = w.sum()
        e1 = (w * E).sum() / Z
        e2 = (w * E * E).sum() / Z
        lnZ = amax + np.log(Z)
        u[i] = e1 / N
        c[i] = (e2 - e1 * e1) / (N * t * t)
        f[i] = -t * lnZ / N
        s[i] = (u[i] - f[i]) / t
    return u, c, f, s


def canonical_distribution(lng, T):
    lng = np.asarray(lng, dtype=np.float64)
    N, E = _energies(lng)
    a = lng - E / T
    out = np.zeros(len(lng))
    ok = np.isfinite(lng)
    out[ok] = np.exp(a[ok] - a[ok].max())
    return out


def specific_heat_peak(lng, T_lo, T_hi, grid=4001):
    from scipy.optimize import minimize_scalar
    Ts = np.linspace(T_lo, T_hi, grid)
    c = canonical(lng, Ts)[1]
    k = int(np.argmax(c))
    lo, hi = Ts[max(k - 1, 0)], Ts[min(k + 1, grid - 1)]
    r = minimize_scalar(lambda t: -canonical(lng, [t])[1][0], bounds=(lo, hi), method="bounded",
                        options={"xatol": 1e-13 * T_hi})
    T = float(r.x)
    cT = float(canonical(lng, [T])[1][0])
    if c[k] > cT:
        T, cT = float(Ts[k]), float(c[k])
    return T, cT


def equal_peak_temperature(lng, T_lo, T_hi):
    """(Tc, E_low, E_high, ln_suppression); None when no pair qualifies."""
    lng = np.asarray(lng, dtype=np.float64)
    N, E = _energies(lng)
    idx = np.flatnonzero(np.isfinite(lng))
    # A bin with no finite ln g (no configuration) is never a maximum.
    lg, Ef = lng[idx], E[idx]
    n = len(idx)
    verts = []
    for i in range(n):
        lower = [(lg[i] - lg[j]) / (Ef[i] - Ef[j]) for j in range(i)]
        higher = [(lg[j] - lg[i]) / (Ef[j] - Ef[i]) for j in range(i + 1, n)]
        beta_max = min(lower) if lower else np.inf     # i beats every lower bin for 1/T <= beta_max
        beta_min = max(higher) if higher else -np.inf  # ... and every higher bin for 1/T >= beta_min
        if beta_min < beta_max:
            verts.append(i)
    best = None
    for a, b in zip(verts[:-1], verts[1:]):
        beta = (lg[b] - lg[a]) / (Ef[b] - Ef[a])
        if beta <= 0:
            continue
        T = 1.0 / beta
        if not (T_lo <= T <= T_hi):
            continue
        width = Ef[b] - Ef[a]
        if best is None or width > best[0]:
            best = (width, T, a, b)
    if best is None:
        return None
    _, T, a, b = best
    between = lg[a:b + 1] - Ef[a:b + 1] / T
    ln_sup = between.min() - (lg[a] - Ef[a] / T)
    return T, int(Ef[a]), int(Ef[b]), float(ln_sup)


def average_pieces(lng_runs, mask_runs, draws):
    """Bin-by-bin mean of the window pieces of runs `draws` over the runs that
    visited the bin; the mask of the mean is 'visited by any'."""
    lw = np.asarray(lng_runs, dtype=np.float64)[list(draws)]
    mw = np.asarray(mask_runs, dtype=np.uint8)[list(draws)]
    cnt = mw.astype(np.int64).sum(axis=0)
    tot = np.where(mw != 0, lw, 0.0).sum(axis=0)
    mean = np.where(cnt > 0, tot / np.maximum(cnt, 1), 0.0)
    return mean, (cnt > 0).astype(np.uint8)


def bootstrap(q, N, e_lo, W, lng_runs, mask_runs, draws):
    """One joined, normalised ln g per row of draws (resample k uses runs draws[k])."""
    out = []
    for row in np.atleast_2d(draws):
        mean, mask = average_pieces(lng_runs, mask_runs, row)
        out.append(_orc.normalise(q, N, _orc.join_pieces(N, e_lo, W, mean, mask)))
    return np.array(out)


def combine_heo(heo, e_lo, N):
    """H(E,O) of the windows (h, W+1, n_obins) summed onto the 2N+1 energies."""
    heo = np.asarray(heo)
    h, B, n_o = heo.shape
    out = np.zeros((2 * N + 1, n_o), dtype=np.uint64)
    for w in range(h):
        b0 = int(e_lo[w]) + 2 * N
        out[b0:b0 + B] += heo[w]
    return out


def canonical_observable(lng, counts, o_values, T):
    """<O>(T) at each temperature of T from ln g and H(E,O) counts (2N+1, n_o)
    whose class o stands for the value o_values[o]."""
    lng = np.asarray(lng, dtype=np.float64)
    N, E = _energies(lng)
    counts = np.asarray(counts, dtype=np.float64)
    tot = counts.sum(axis=1)
    ok = np.isfinite(lng) & (tot > 0)
    o_mean = (counts[ok] * np.asarray(o_values, dtype=np.float64)[None, :]).sum(axis=1) / tot[ok]
    out = []
    for t in np.atleast_1d(T):
        a = lng[ok] - E[ok] / t
        w = np.exp(a - a.max())
        out.append((w * o_mean).sum() / w.sum())
    return np.array(out)
