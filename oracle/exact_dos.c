/*
 * exact_dos.c -- exact densities of states of the periodic 2D q-state Potts
 * model (Eq. 2), used to pin the REWL oracle.  TEST INFRASTRUCTURE ONLY.
 *
 * Counts are indexed by the number of unsatisfied ("broken") bonds
 * b = E + 2N in [0, 2N], with E = -(number of satisfied bonds).
 *
 *   ex_brute_force     : every one of the q^N configurations, bonds counted
 *                        one by one (small cases only).
 *   ex_transfer_matrix : the same counts by adding one site at a time to a
 *                        frontier of the last L spins, with the first row held
 *                        fixed so that the periodic bonds can be closed at the
 *                        end.  Optionally only one first row per colour-
 *                        permutation class is propagated and weighted by the
 *                        class size.  Exact in unsigned 128-bit integers.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

static int bond_broken(const uint8_t *s, int a, int b) { return s[a] != s[b]; }

int ex_brute_force(int q, int L, uint64_t *counts)
{
    int N = L * L;
    double states = 1.0;
    for (int i = 0; i < N; ++i) states *= q;
    if (L < 3 || q < 2 || states > 1.5e9) return 1;
    memset(counts, 0, sizeof(uint64_t) * (size_t)(2 * N + 1));
    uint8_t *s = (uint8_t *)calloc((size_t)N, 1);
    for (;;) {
        int broken = 0;
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int i = y * L + x;
                broken += bond_broken(s, i, y * L + (x + 1) % L);
                broken += bond_broken(s, i, ((y + 1) % L) * L + x);
            }
        counts[broken] += 1;
        int pos = 0; /* odometer increment */
        while (pos < N && ++s[pos] == q) s[pos++] = 0;
        if (pos == N) break;
    }
    free(s);
    return 0;
}

/* digit i of a base-q frontier code */
static int digit(uint32_t code, int i, const uint32_t *pw, int q) { return (int)((code / pw[i]) % (uint32_t)q); }

/* Restricted growth test: colours appear in first-occurrence order 0, 1, 2...
 * Returns the number of distinct colours, or 0 if the row is not canonical. */
static int canonical_colours(uint32_t code, int L, const uint32_t *pw, int q)
{
    int mx = -1;
    for (int i = 0; i < L; ++i) {
        int d = digit(code, i, pw, q);
        if (d > mx + 1) return 0;
        if (d > mx) mx = d;
    }
    return mx + 1;
}

int ex_transfer_matrix(int q, int L, int use_symmetry, uint64_t *hi, uint64_t *lo)
{
    if (q < 2 || L < 3) return 1;
    int N = L * L, P = 2 * N + 1;
    double nst_d = 1.0;
    for (int i = 0; i < L; ++i) nst_d *= q;
    if (nst_d > 2.0e6) return 1;
    uint32_t nst = (uint32_t)nst_d;
    uint32_t pw[32];
    pw[0] = 1;
    for (int i = 1; i <= L; ++i) pw[i] = pw[i - 1] * (uint32_t)q;
    u128 *cur = (u128 *)calloc((size_t)nst * P, sizeof(u128));
    u128 *nxt = (u128 *)calloc((size_t)nst * P, sizeof(u128));
    u128 *total = (u128 *)calloc((size_t)P, sizeof(u128));
    uint8_t *live = (uint8_t *)calloc(nst, 1), *nlive = (uint8_t *)calloc(nst, 1);
    if (!cur || !nxt || !total || !live || !nlive) return 2;

    for (uint32_t s0 = 0; s0 < nst; ++s0) {
        u128 weight = 1;
        if (use_symmetry) {
            int c = canonical_colours(s0, L, pw, q);
            if (!c) continue;
            for (int i = 0; i < c; ++i) weight *= (u128)(q - i);
        }
        memset(cur, 0, sizeof(u128) * (size_t)nst * P);
        memset(live, 0, nst);
        int b0 = 0; /* row 0, horizontal bonds including the periodic one */
        for (int x = 0; x < L; ++x) b0 += digit(s0, x, pw, q) != digit(s0, (x + 1) % L, pw, q);
        cur[(size_t)s0 * P + b0] = 1;
        live[s0] = 1;
        for (int y = 1; y < L; ++y) {
            for (int x = 0; x < L; ++x) {
                memset(nxt, 0, sizeof(u128) * (size_t)nst * P);
                memset(nlive, 0, nst);
                for (uint32_t st = 0; st < nst; ++st) {
                    if (!live[st]) continue;
                    int up = digit(st, 0, pw, q);
                    int left = digit(st, L - 1, pw, q);
                    int first = digit(st, 1, pw, q); /* site (0, y) when x = L-1 */
                    for (int c = 0; c < q; ++c) {
                        int add = (c != up);
                        if (x > 0) add += (c != left);
                        if (x == L - 1) add += (c != first);
                        uint32_t ns = st / (uint32_t)q + (uint32_t)c * pw[L - 1];
                        const u128 *src = cur + (size_t)st * P;
                        u128 *dst = nxt + (size_t)ns * P + add;
                        for (int k = 0; k + add < P; ++k) dst[k] += src[k];
                        nlive[ns] = 1;
                    }
                }
                u128 *tmp = cur; cur = nxt; nxt = tmp;
                uint8_t *tl = live; live = nlive; nlive = tl;
            }
        }
        for (uint32_t st = 0; st < nst; ++st) { /* close the vertical periodic bonds */
            if (!live[st]) continue;
            int add = 0;
            for (int i = 0; i < L; ++i) add += digit(st, i, pw, q) != digit(s0, i, pw, q);
            for (int k = 0; k + add < P; ++k) total[k + add] += weight * cur[(size_t)st * P + k];
        }
    }
    for (int k = 0; k < P; ++k) {
        hi[k] = (uint64_t)(total[k] >> 64);
        lo[k] = (uint64_t)total[k];
    }
    free(cur); free(nxt); free(total); free(live); free(nlive);
    return 0;
}
