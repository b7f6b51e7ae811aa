// rewl_analysis.cu -- analysis of densities of states behind include/rewl.h:
// canonical averages and the canonical distribution (Sec. 3.1, Fig. 3b), the
// specific-heat maximum, the equal-peak finite-size transition temperature
// with the suppression of the transition states (Sec. 3.1), the join of
// caller-supplied window pieces, and bootstrap resampling of repeated runs
// (end of Sec. 2).  Host code: these act on at most 2N + 1 bins once per run,
// after the sampling the GPU does.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "rewl.h"
#include "rewl_host_internal.hpp"

using rewl::host::fail;

namespace {

// 2N + 1 bins, E = b - 2N.  Finite ln g required somewhere; +inf / NaN refused.
rewl_status check_lng(const double *lng, size_t len, int *N) {
    if (!lng) return fail(REWL_ERR_ARG, "NULL ln g");
    if (len < 3 || len % 2 == 0 || len > (size_t)8 * 1024 * 1024 + 1)
        return fail(REWL_ERR_ARG, "ln g length %zu is not 2N + 1 for a supported N", len);
    bool any = false;
    for (size_t b = 0; b < len; ++b) {
        if (std::isnan(lng[b]) || lng[b] == INFINITY) return fail(REWL_ERR_ARG, "ln g[%zu] is NaN or +inf", b);
        any = any || lng[b] != -INFINITY;
    }
    if (!any) return fail(REWL_ERR_ARG, "ln g has no finite bin");
    *N = (int)((len - 1) / 2);
    return REWL_OK;
}

bool bad_temperature(double T) { return !(T > 0.0) || !std::isfinite(T); }

// The finite bins as (E, ln g) pairs in increasing E.
struct Bins {
    std::vector<double> E, lg;
    Bins(const double *lng, size_t len, int N) {
        for (size_t b = 0; b < len; ++b)
            if (lng[b] != -INFINITY) {
                E.push_back((double)b - 2.0 * N);
                lg.push_back(lng[b]);
            }
    }
};

struct Moments {
    double u, c, f, s;
};

// Canonical averages at T over the bins, weights g(E) exp(-E/T) scaled by the
// largest one (each computed once, in `w`); the variance is taken about the
// mean (no cancellation).
Moments moments(const Bins &x, int N, double T, std::vector<double> &w) {
    const size_t n = x.E.size();
    w.resize(n);
    double top = -INFINITY;
    for (size_t i = 0; i < n; ++i) top = std::fmax(top, x.lg[i] - x.E[i] / T);
    double Z = 0.0, e1 = 0.0;
    for (size_t i = 0; i < n; ++i) {
        w[i] = std::exp((x.lg[i] - x.E[i] / T) - top);
        Z += w[i];
        e1 += w[i] * x.E[i];
    }
    e1 /= Z;
    double var = 0.0;
    for (size_t i = 0; i < n; ++i) {
        const double d = x.E[i] - e1;
        var += w[i] * d * d;
    }
    var /= Z;
    Moments m;
    m.u = e1 / N;
    m.c = var / ((double)N * T * T);
    m.f = -T * (top + std::log(Z)) / N;
    m.s = (m.u - m.f) / T;
    return m;
}

}  // namespace

extern "C" {

rewl_status rewl_canonical(const double *lng, size_t len, const double *T, size_t nT, double *out) {
    REWL_API_TRY
    int N;
    rewl_status st = check_lng(lng, len, &N);
    if (st) return st;
    if ((nT && (!T || !out))) return fail(REWL_ERR_ARG, "NULL temperatures or output");
    for (size_t i = 0; i < nT; ++i)
        if (bad_temperature(T[i])) return fail(REWL_ERR_ARG, "temperature %zu is not finite and > 0", i);
    const Bins x(lng, len, N);
    std::vector<double> w;
    for (size_t i = 0; i < nT; ++i) {
        const Moments m = moments(x, N, T[i], w);
        out[4 * i + 0] = m.u;
        out[4 * i + 1] = m.c;
        out[4 * i + 2] = m.f;
        out[4 * i + 3] = m.s;
    }
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_canonical_distribution(const double *lng, size_t len, double T, double *out) {
    REWL_API_TRY
    int N;
    rewl_status st = check_lng(lng, len, &N);
    if (st) return st;
    if (!out) return fail(REWL_ERR_ARG, "NULL output");
    if (bad_temperature(T)) return fail(REWL_ERR_ARG, "temperature is not finite and > 0");
    double top = -INFINITY;
    for (size_t b = 0; b < len; ++b)
        if (lng[b] != -INFINITY) top = std::fmax(top, lng[b] - ((double)b - 2.0 * N) / T);
    for (size_t b = 0; b < len; ++b)
        out[b] = lng[b] == -INFINITY ? 0.0 : std::exp((lng[b] - ((double)b - 2.0 * N) / T) - top);
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_specific_heat_peak(const double *lng, size_t len, double T_lo, double T_hi, double *T_peak,
                                    double *c_peak) {
    REWL_API_TRY
    int N;
    rewl_status st = check_lng(lng, len, &N);
    if (st) return st;
    if (!T_peak || !c_peak) return fail(REWL_ERR_ARG, "NULL output");
    if (bad_temperature(T_lo) || !std::isfinite(T_hi) || !(T_hi > T_lo))
        return fail(REWL_ERR_ARG, "temperature range [%g, %g] invalid", T_lo, T_hi);
    const Bins x(lng, len, N);
    std::vector<double> w;
    auto c_at = [&](double T) { return moments(x, N, T, w).c; };
    // Scan, then golden-section search between the best point's neighbours.
    const int grid = 1024;
    const double step = (T_hi - T_lo) / grid;
    int k_best = 0;
    double c_best = -1.0;
    for (int k = 0; k <= grid; ++k) {
        const double c = c_at(k == grid ? T_hi : T_lo + k * step);
        if (c > c_best) {
            c_best = c;
            k_best = k;
        }
    }
    double a = T_lo + (k_best > 0 ? k_best - 1 : 0) * step;
    double b = k_best + 1 < grid ? T_lo + (k_best + 1) * step : T_hi;
    const double r = 0.5 * (std::sqrt(5.0) - 1.0);
    double x1 = b - r * (b - a), x2 = a + r * (b - a);
    double c1 = c_at(x1), c2 = c_at(x2);
    for (int it = 0; it < 200 && (b - a) > 1e-13 * T_hi; ++it) {
        if (c1 >= c2) {
            b = x2;
            x2 = x1;
            c2 = c1;
            x1 = b - r * (b - a);
            c1 = c_at(x1);
        } else {
            a = x1;
            x1 = x2;
            c1 = c2;
            x2 = a + r * (b - a);
            c2 = c_at(x2);
        }
    }
    double T = c1 >= c2 ? x1 : x2, c = c1 >= c2 ? c1 : c2;
    if (c_best > c) {
        T = k_best == grid ? T_hi : T_lo + k_best * step;
        c = c_best;
    }
    *T_peak = T;
    *c_peak = c;
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_equal_peak_temperature(const double *lng, size_t len, double T_lo, double T_hi, double *Tc,
                                        int *e_low, int *e_high, double *ln_suppression) {
    REWL_API_TRY
    int N;
    rewl_status st = check_lng(lng, len, &N);
    if (st) return st;
    if (!Tc) return fail(REWL_ERR_ARG, "NULL output");
    if (bad_temperature(T_lo) || !(T_hi >= T_lo)) return fail(REWL_ERR_ARG, "temperature range [%g, %g] invalid", T_lo, T_hi);
    const Bins x(lng, len, N);
    const size_t n = x.E.size();
    auto slope = [&](size_t i, size_t j) { return (x.lg[j] - x.lg[i]) / (x.E[j] - x.E[i]); };
    // Upper concave hull of (E, ln g), scanned in increasing E: the last vertex
    // is dropped while it lies on or under the segment from the one before it
    // to the new bin.  Successive hull vertices are exactly the pairs of bins
    // that are both maxima of ln g(E) - E/T at T = 1 / slope.
    std::vector<size_t> hull;
    for (size_t i = 0; i < n; ++i) {
        while (hull.size() >= 2 && slope(hull[hull.size() - 2], hull.back()) <= slope(hull.back(), i)) hull.pop_back();
        hull.push_back(i);
    }
    bool found = false;
    double best_w = 0.0, best_T = 0.0;
    size_t best_a = 0, best_b = 0;
    for (size_t k = 0; k + 1 < hull.size(); ++k) {
        const size_t a = hull[k], b = hull[k + 1];
        const double beta = slope(a, b);
        if (!(beta > 0.0)) continue;
        const double T = 1.0 / beta;
        if (!(T_lo <= T && T <= T_hi)) continue;
        const double w = x.E[b] - x.E[a];
        if (!found || w > best_w) {
            found = true;
            best_w = w;
            best_T = T;
            best_a = a;
            best_b = b;
        }
    }
    if (!found) return fail(REWL_ERR_STATE, "no pair of equal canonical peaks with T in [%g, %g]", T_lo, T_hi);
    double low = INFINITY;
    for (size_t i = best_a; i <= best_b; ++i) low = std::fmin(low, x.lg[i] - x.E[i] / best_T);
    *Tc = best_T;
    if (e_low) *e_low = (int)x.E[best_a];
    if (e_high) *e_high = (int)x.E[best_b];
    if (ln_suppression) *ln_suppression = low - (x.lg[best_a] - x.E[best_a] / best_T);
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_ising_energy(int L, int b, long long *e_ising) {
    REWL_API_TRY
    if (!e_ising) return fail(REWL_ERR_ARG, "NULL output");
    if (L < 3 || L > 1024) return fail(REWL_ERR_ARG, "L=%d outside [3, 1024]", L);
    const long long N = (long long)L * L;
    if (b < 0 || b > 2 * N) return fail(REWL_ERR_ARG, "bin %d outside [0, 2N]", b);
    *e_ising = 2LL * b - 2LL * N;
    return REWL_OK;
    REWL_API_CATCH
}

}  // extern "C"

namespace {

rewl_status check_pieces(int q, int L, int h, int W, const int *e_lo, size_t len) {
    if (q < 2 || q > 255) return fail(REWL_ERR_ARG, "q=%d outside [2, 255]", q);
    if (L < 3 || L > 1024) return fail(REWL_ERR_ARG, "L=%d outside [3, 1024]", L);
    const int N = L * L;
    if (h < 1 || W < 1 || W > 2 * N) return fail(REWL_ERR_ARG, "h=%d or W=%d out of range", h, W);
    if (!e_lo) return fail(REWL_ERR_ARG, "NULL window table");
    for (int a = 0; a < h; ++a) {
        if (e_lo[a] < -2 * N || e_lo[a] + W > 0) return fail(REWL_ERR_ARG, "window %d leaves [-2N, 0]", a);
        if (a && e_lo[a] < e_lo[a - 1]) return fail(REWL_ERR_ARG, "window table not increasing at %d", a);
    }
    if (len != (size_t)(2 * N + 1)) return fail(REWL_ERR_ARG, "len %zu != 2N + 1 = %d", len, 2 * N + 1);
    return REWL_OK;
}

}  // namespace

extern "C" {

rewl_status rewl_join(int q, int L, int h, int W, const int *e_lo, const double *lng_w, const unsigned char *mask_w,
                      double *out, size_t len) {
    REWL_API_TRY
    rewl_status st = check_pieces(q, L, h, W, e_lo, len);
    if (st) return st;
    if (!lng_w || !mask_w || !out) return fail(REWL_ERR_ARG, "NULL argument");
    const size_t n = (size_t)h * (W + 1);
    std::vector<int32_t> el(e_lo, e_lo + h);
    std::vector<double> lw(lng_w, lng_w + n);
    std::vector<uint8_t> mw(mask_w, mask_w + n);
    const int N = L * L;
    st = rewl::host::join_windows(N, W, el, lw, mw, out);
    if (st) return st;
    rewl::host::normalise_total(q, N, out, 2 * N + 1);
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_bootstrap(int q, int L, int h, int W, const int *e_lo, int runs, const double *lng_runs,
                           const unsigned char *mask_runs, int resamples, const int *draws, double *out, size_t len) {
    REWL_API_TRY
    rewl_status st = check_pieces(q, L, h, W, e_lo, len);
    if (st) return st;
    if (runs < 1 || resamples < 0) return fail(REWL_ERR_ARG, "runs=%d or resamples=%d out of range", runs, resamples);
    if (resamples && (!lng_runs || !mask_runs || !draws || !out)) return fail(REWL_ERR_ARG, "NULL argument");
    for (long long k = 0; k < (long long)resamples * runs; ++k)
        if (draws[k] < 0 || draws[k] >= runs) return fail(REWL_ERR_ARG, "draw %lld names run %d of %d", k, draws[k], runs);
    const int N = L * L;
    const size_t n = (size_t)h * (W + 1);
    std::vector<int32_t> el(e_lo, e_lo + h);
    std::vector<double> sum(n);
    std::vector<int> cnt(n);
    std::vector<uint8_t> mask(n);
    for (int k = 0; k < resamples; ++k) {
        std::fill(sum.begin(), sum.end(), 0.0);
        std::fill(cnt.begin(), cnt.end(), 0);
        for (int r = 0; r < runs; ++r) {
            const size_t run = (size_t)draws[(size_t)k * runs + r];
            const double *lg = lng_runs + run * n;
            const unsigned char *mk = mask_runs + run * n;
            for (size_t i = 0; i < n; ++i)
                if (mk[i]) {
                    sum[i] += lg[i];
                    ++cnt[i];
                }
        }
        for (size_t i = 0; i < n; ++i) {
            mask[i] = cnt[i] > 0;
            sum[i] = cnt[i] > 0 ? sum[i] / cnt[i] : 0.0;
        }
        double *o = out + (size_t)k * len;
        st = rewl::host::join_windows(N, W, el, sum, mask, o);
        if (st) return st;
        rewl::host::normalise_total(q, N, o, 2 * N + 1);
    }
    return REWL_OK;
    REWL_API_CATCH
}

}  // extern "C"
