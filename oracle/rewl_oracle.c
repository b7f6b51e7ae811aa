/*
 * rewl_oracle.c -- plain, single-threaded CPU oracle for Replica-Exchange
 * Wang-Landau (REWL) sampling of the periodic 2D q-state Potts model.
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA path.  Only the
 * test suite, the package smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header or constant table with the CUDA library.
 *
 * Source: Vogel, Li, Wuest & Landau, "Exploring new frontiers in statistical
 * physics with a new, parallel Wang-Landau framework" (arXiv:1312.3004).
 *   Sec. 2   : the REWL scheme (energy windows, m walkers per window, flatness
 *              of every walker, averaging of g inside a window, f -> sqrt(f),
 *              replica exchange with Eq. 1, joining of the pieces, Fig. 2).
 *   Eq. 2    : Potts Hamiltonian H = -sum_<ij> delta(s_i, s_j), N = L x L.
 *   Sec. 3.1 : single-spin-flip updates; 717 windows / 75% overlap for L=300.
 *
 * Where the paper is silent, the readings below are the ones this project
 * fixes for both the oracle and the CUDA path (written independently):
 *   - periodic boundaries; site s = y*L + x; E in [-2N, 0]; bin b = E + 2N;
 *   - equal windows: R = 2N, W = ceil(R / (1 + (h-1)(1-o))), W+1 bins each,
 *     E_lo(i) = -2N + round_half_up(i (R-W) / (h-1));
 *   - random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed,
 *     counter = (c0, c1, c2, domain) with the domain table below;
 *   - WL step: site = r0*N >> 32, new spin uniform over the q-1 other values,
 *     proposals leaving the window are rejected, accept iff D >= 0 or
 *     u < exp(D) with D = ln g(E_old) - ln g(E_new), then ln g(E) += ln f and
 *     H(E) += 1 at the (possibly unchanged) current energy;
 *   - barrier every K steps: visited mask, flatness min >= p * mean over the
 *     mask, merge = pairwise-tree mean of ln g, ln f -> ln f / 2, done when
 *     ln f < ln f_final, then replica exchange between windows (a, a+1) with
 *     a = round mod 2 and a random one-to-one matching of the m walkers;
 *   - joining at the bin where the two pieces' central-difference slopes
 *     agree best; normalisation sum_E g(E) = q^N;
 *   - optional ln f schedule: the 1/t rule (Belardinelli & Pereyra), which
 *     Sec. 2 admits as another valid WL update rule (orc_window_iterations);
 *   - optional fixed-weight production with ln f = 0 and a histogram H(E,O)
 *     of the majority count O (Sec. 3.2's production runs), orc_production_*.
 *
 * Floating point: IEEE binary64, round to nearest, no contraction (build with
 * -ffp-contract=off).  exp/log come from the C library.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, from the definition in Salmon, Moraes, Dror & Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64
 * multiplications whose halves are crossed with the other counter words and
 * the round key; the key is bumped by the two Weyl constants between rounds. */
#define ORC_PHILOX_MUL0 0xD2511F53u
#define ORC_PHILOX_MUL1 0xCD9E8D57u
#define ORC_PHILOX_WEYL0 0x9E3779B9u
#define ORC_PHILOX_WEYL1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_WEYL0;
            k1 += ORC_PHILOX_WEYL1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_MUL0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_MUL1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Random-number domains (fourth counter word). */
enum {
    ORC_DOM_WL = 0,    /* c0,c1 = WL step t (lo, hi), c2 = global walker index */
    ORC_DOM_INIT = 1,  /* c0 = site / 4, c1 = 0, c2 = walker: initial spins      */
    ORC_DOM_ENTRY = 2, /* c0,c1 = entry proposal n, c2 = walker                   */
    ORC_DOM_PERM = 3,  /* c0 = round, c1 = word / 4, c2 = lower window a          */
    ORC_DOM_XACC = 4   /* c0 = round, c1 = pair k, c2 = lower window a            */
};

static void orc_draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t dom,
                     uint32_t r[4])
{
    uint32_t ctr[4] = {c0, c1, c2, dom};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, r);
}

/* Uniform integer in [0, n) by the multiply-shift map (not modulo). */
static uint32_t orc_below(uint32_t word, uint32_t n)
{
    return (uint32_t)(((uint64_t)word * (uint64_t)n) >> 32);
}

/* Uniform double in [0, 1) with 53 random bits: 27 from hi, 26 from lo. */
static double orc_u53(uint32_t hi, uint32_t lo)
{
    uint64_t bits = ((uint64_t)(hi >> 5) << 26) | (uint64_t)(lo >> 6);
    return (double)bits * 0x1p-53;
}

/* Decision bookkeeping for the GPU comparison (test support, no effect on a
 * run unless a test asks for it).  A draw with |u - exp(d)| below
 * ORC_TIE_NEAR is logged: two libraries' exp can decide such a draw
 * differently.  A test can also ask for given decisions to be inverted, to
 * reproduce what another implementation did at a near tie.  Decisions are
 * named by (kind, who, when): kind 0 a WL step of walker `who` at its step
 * index `when`; kind 1 the exchange of the pair whose lower-window walker is
 * `who`, in round `when`. */
#define ORC_TIE_NEAR 1e-12
#define ORC_TIE_LOG 64
#define ORC_MAX_INVERT 16
typedef struct orc_decisions {
    int n_invert;
    uint64_t invert[ORC_MAX_INVERT][3];
    int64_t n_wl, n_wl_neg;              /* WL decisions made; those with d < 0 */
    int64_t n_ties;                      /* near-tie draws seen (all of them)   */
    uint64_t tie[ORC_TIE_LOG][3];        /* first ORC_TIE_LOG: kind, who, when */
    double tie_gap[ORC_TIE_LOG];         /* |u - exp(d)| of each               */
} orc_decisions;

/* ------------------------------------------------------------------------- */
/* Energy windows (Sec. 2, Fig. 1; geometry pinned by the L=300 run of Sec. 3.1:
 * 717 windows with 75% overlap give W = 1000 and a stride of 250 bins). */
int orc_window_table(int L, int h, double overlap, int32_t *e_lo, int32_t *W_out)
{
    if (L < 3 || h < 1 || !(overlap >= 0.0 && overlap < 1.0)) return 1;
    int64_t N = (int64_t)L * L;
    int64_t R = 2 * N;
    double denom = 1.0 + (double)(h - 1) * (1.0 - overlap);
    int64_t W = (int64_t)ceil((double)R / denom);
    if (W > R) W = R;
    if (W < 8) return 1;
    for (int i = 0; i < h; ++i) {
        int64_t off = 0;
        if (h > 1) off = (2 * (int64_t)i * (R - W) + (h - 1)) / (2 * (int64_t)(h - 1));
        if (e_lo) e_lo[i] = (int32_t)(-2 * N + off);
    }
    *W_out = (int32_t)W;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Potts model (Eq. 2), periodic square lattice. */
static int orc_nbr(int L, int s, int dir)
{
    int x = s % L, y = s / L;
    switch (dir) {
    case 0: x = (x + 1) % L; break;
    case 1: x = (x + L - 1) % L; break;
    case 2: y = (y + 1) % L; break;
    default: y = (y + L - 1) % L; break;
    }
    return y * L + x;
}

/* E = -(number of satisfied bonds); each site owns its right and down bond. */
int32_t orc_energy(int L, const uint8_t *sigma)
{
    int N = L * L;
    int32_t sat = 0;
    for (int s = 0; s < N; ++s) {
        sat += sigma[s] == sigma[orc_nbr(L, s, 0)];
        sat += sigma[s] == sigma[orc_nbr(L, s, 2)];
    }
    return -sat;
}

/* Energy change of setting site s from cur to nw. */
static int orc_delta_e(int L, const uint8_t *sigma, int s, int cur, int nw)
{
    int d = 0;
    for (int dir = 0; dir < 4; ++dir) {
        int sn = sigma[orc_nbr(L, s, dir)];
        d += (sn == cur) - (sn == nw);
    }
    return d;
}

/* ------------------------------------------------------------------------- */
typedef struct orc_rewl {
    int q, L, N, h, m, W;
    double overlap, lnf_final, flatness;
    int64_t K;
    uint64_t seed;
    int32_t *e_lo;   /* [h] lowest energy of window i; window spans W+1 bins */
    uint8_t *sigma;  /* [h*m][N] configuration carried by walker g = i*m + k */
    int32_t *E;      /* [h*m] energy of that configuration                    */
    uint32_t *rep;   /* [h*m] replica id of that configuration                */
    uint64_t *t;     /* [h*m] WL steps made by walker g                        */
    double *lng;     /* [h*m][W+1] ln g estimate of walker g                   */
    uint32_t *H;     /* [h*m][W+1] histogram of walker g, current iteration    */
    uint8_t *mask;   /* [h][W+1] bins visited by any walker of the window     */
    double *lnf;     /* [h] ln f of window i                                  */
    int32_t *iter;   /* [h] completed WL iterations of window i              */
    uint8_t *done;   /* [h] 1 once ln f < ln f_final                          */
    uint8_t *rt_end; /* [h*m] by replica id: last end of the energy range the
                        replica's window touched (0 none yet, 1 lowest window,
                        2 highest window)                                      */
    uint32_t *rt_trips; /* [h*m] by replica id: completed round trips, lowest
                        window -> highest -> lowest                            */
    int schedule;    /* ln f schedule: 0 halving (Sec. 2), 1 the 1/t rule     */
    uint8_t *phase;  /* [h] 1/t rule: 1 once the window follows ln f = 1/t   */
    int production;  /* 1: fixed-weight production (ln f = 0, H(E,O) kept)   */
    int n_obins;     /* classes of the observable O = majority count         */
    uint64_t *heo;   /* [h][W+1][n_obins] production histogram H(E,O)        */
    int64_t round;   /* barriers (exchange rounds) completed                  */
    uint64_t xtried, xacc;
    int status;
    orc_decisions dec; /* near-tie log and inverted decisions (test support) */
} orc_rewl;

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_NOMEM = 2, ORC_ERR_OVERFLOW = 5, ORC_ERR_STATE = 6 };

/* Metropolis-type acceptance with ratio exp(d), i.e. min[1, exp(d)] (Sec. 2;
 * Eq. 1 for an exchange): accept iff d >= 0 or u < exp(d); plus the
 * bookkeeping above. */
static int orc_decide(orc_rewl *s, int kind, uint64_t who, uint64_t when, double d, double u)
{
    int acc = 1;
    if (kind == 0) {
        s->dec.n_wl += 1;
        s->dec.n_wl_neg += d < 0.0;
    }
    if (d < 0.0) {
        double e = exp(d);
        double gap = fabs(u - e);
        acc = u < e;
        if (gap < ORC_TIE_NEAR) {
            if (s->dec.n_ties < ORC_TIE_LOG) {
                uint64_t *ent = s->dec.tie[s->dec.n_ties];
                ent[0] = (uint64_t)kind; ent[1] = who; ent[2] = when;
                s->dec.tie_gap[s->dec.n_ties] = gap;
            }
            s->dec.n_ties += 1;
        }
    }
    for (int i = 0; i < s->dec.n_invert; ++i) {
        const uint64_t *e = s->dec.invert[i];
        if (e[0] == (uint64_t)kind && e[1] == who && e[2] == when) acc = !acc;
    }
    return acc;
}

int orc_invert_decision(orc_rewl *s, int kind, uint64_t who, uint64_t when)
{
    if (s->dec.n_invert >= ORC_MAX_INVERT) return ORC_ERR_ARG;
    uint64_t *e = s->dec.invert[s->dec.n_invert++];
    e[0] = (uint64_t)kind; e[1] = who; e[2] = when;
    return ORC_OK;
}

/* WL acceptance decisions so far (proposals inside the window) and how many
 * of them had d < 0, i.e. needed exp(d). */
void orc_get_decision_counts(const orc_rewl *s, int64_t out[2])
{
    out[0] = s->dec.n_wl;
    out[1] = s->dec.n_wl_neg;
}

/* Near-tie log: returns the number of near ties seen; fills up to `cap`
 * entries (kind, who, when) and their gaps |u - exp(d)|. */
int64_t orc_get_ties(const orc_rewl *s, uint64_t *entries, double *gaps, int cap)
{
    int n = s->dec.n_ties < ORC_TIE_LOG ? (int)s->dec.n_ties : ORC_TIE_LOG;
    if (n > cap) n = cap;
    for (int i = 0; i < n; ++i) {
        entries[3 * i] = s->dec.tie[i][0];
        entries[3 * i + 1] = s->dec.tie[i][1];
        entries[3 * i + 2] = s->dec.tie[i][2];
        gaps[i] = s->dec.tie_gap[i];
    }
    return s->dec.n_ties;
}


void orc_destroy(orc_rewl *s)
{
    if (!s) return;
    free(s->e_lo); free(s->sigma); free(s->E); free(s->rep); free(s->t);
    free(s->lng); free(s->H); free(s->mask); free(s->lnf); free(s->iter); free(s->done);
    free(s->rt_end); free(s->rt_trips); free(s->phase); free(s->heo);
    free(s);
}

/* Replica diffusion through the windows (the quantity REWL's exchanges are
 * there to speed up, Sec. 2): after every exchange round, a replica held by a
 * walker of the lowest window completes a round trip if it has been in the
 * highest window since it last was in the lowest one.  With one window there
 * are no round trips.  Replica c is held by walker g when rep[g] = c. */
void orc_track_round_trips(orc_rewl *s)
{
    size_t G = (size_t)s->h * s->m;
    if (s->h < 2) return;
    for (size_t g = 0; g < G; ++g) {
        uint32_t c = s->rep[g];
        int w = (int)(g / (size_t)s->m);
        if (w == 0) {
            if (s->rt_end[c] == 2) s->rt_trips[c] += 1;
            s->rt_end[c] = 1;
        } else if (w == s->h - 1) {
            s->rt_end[c] = 2;
        }
    }
}

/* Start of the run (Sec. 3.2 describes the same set-up: each walker is handed a
 * configuration whose energy lies inside its window).  Spins are drawn from the
 * seed; a walker whose window lies below that energy restarts from a uniform
 * ground state; it then climbs by single flips that never lower E and never
 * leave the window from above, until E >= E_lo.  Entry moves touch neither
 * ln g nor H. */
static int orc_enter_window(orc_rewl *s, int g)
{
    int N = s->N, q = s->q, L = s->L;
    uint8_t *sg = s->sigma + (size_t)g * N;
    int w = g / s->m;
    int32_t lo = s->e_lo[w], hi = lo + s->W;
    uint32_t r[4];
    for (int site = 0; site < N; ++site) {
        if ((site & 3) == 0) orc_draw(s->seed, (uint32_t)(site >> 2), 0, (uint32_t)g, ORC_DOM_INIT, r);
        sg[site] = (uint8_t)orc_below(r[site & 3], (uint32_t)q);
    }
    int32_t E = orc_energy(L, sg);
    if (E > hi) {
        orc_draw(s->seed, 0, 0, (uint32_t)g, ORC_DOM_ENTRY, r);
        uint8_t c = (uint8_t)orc_below(r[0], (uint32_t)q);
        memset(sg, c, (size_t)N);
        E = -2 * N;
    }
    uint64_t max_moves = 1000ull * (uint64_t)N + 1000000ull;
    for (uint64_t n = 1; E < lo; ++n) {
        if (n > max_moves) return ORC_ERR_STATE;
        orc_draw(s->seed, (uint32_t)n, (uint32_t)(n >> 32), (uint32_t)g, ORC_DOM_ENTRY, r);
        int site = (int)orc_below(r[0], (uint32_t)N);
        int cur = sg[site];
        int v = (int)orc_below(r[1], (uint32_t)(q - 1));
        int nw = v + (v >= cur);
        int32_t En = E + orc_delta_e(L, sg, site, cur, nw);
        if (En >= E && En <= hi) {
            sg[site] = (uint8_t)nw;
            E = En;
        }
    }
    s->E[g] = E;
    return ORC_OK;
}

orc_rewl *orc_create(int q, int L, int h, double overlap, int m, double lnf_final,
                     double flatness, int64_t K, uint64_t seed, int *status)
{
    *status = ORC_ERR_ARG;
    if (q < 2 || q > 255 || L < 3 || L > 4096 || h < 1 || m < 1 || K < 1) return NULL;
    if (!(lnf_final > 0.0 && lnf_final < 1.0) || !(flatness > 0.0 && flatness < 1.0)) return NULL;
    int32_t W;
    if (orc_window_table(L, h, overlap, NULL, &W)) return NULL;
    orc_rewl *s = (orc_rewl *)calloc(1, sizeof(orc_rewl));
    *status = ORC_ERR_NOMEM;
    if (!s) return NULL;
    s->q = q; s->L = L; s->N = L * L; s->h = h; s->m = m; s->W = W;
    s->overlap = overlap; s->lnf_final = lnf_final; s->flatness = flatness;
    s->K = K; s->seed = seed;
    size_t G = (size_t)h * m, B = (size_t)W + 1;
    s->e_lo = calloc((size_t)h, sizeof(int32_t));
    s->sigma = calloc(G * (size_t)s->N, 1);
    s->E = calloc(G, sizeof(int32_t));
    s->rep = calloc(G, sizeof(uint32_t));
    s->t = calloc(G, sizeof(uint64_t));
    s->lng = calloc(G * B, sizeof(double));
    s->H = calloc(G * B, sizeof(uint32_t));
    s->mask = calloc((size_t)h * B, 1);
    s->lnf = calloc((size_t)h, sizeof(double));
    s->iter = calloc((size_t)h, sizeof(int32_t));
    s->done = calloc((size_t)h, 1);
    s->rt_end = calloc(G, 1);
    s->rt_trips = calloc(G, sizeof(uint32_t));
    s->phase = calloc((size_t)h, 1);
    if (!s->e_lo || !s->sigma || !s->E || !s->rep || !s->t || !s->lng || !s->H || !s->mask ||
        !s->lnf || !s->iter || !s->done || !s->rt_end || !s->rt_trips || !s->phase) {
        orc_destroy(s);
        return NULL;
    }
    orc_window_table(L, h, overlap, s->e_lo, &W);
    for (int i = 0; i < h; ++i) s->lnf[i] = 1.0; /* ln f_0 = 1, i.e. f_0 = e */
    for (size_t g = 0; g < G; ++g) {
        s->rep[g] = (uint32_t)g;
        int st = orc_enter_window(s, (int)g);
        if (st) {
            orc_destroy(s);
            *status = st;
            return NULL;
        }
    }
    orc_track_round_trips(s); /* the replicas' starting windows */
    *status = ORC_OK;
    return s;
}

/* ------------------------------------------------------------------------- */
/* n standard WL steps of walker g at its window's ln f (Sec. 2, standard WL
 * paragraph; single-spin-flip proposals of Sec. 3.1). */
/* The Potts observable of the production run: the majority count
 * n_max = max over k of #{i : s_i = k}, in [ceil(N/q), N]. */
int orc_majority(const uint8_t *sigma, int N, int q)
{
    int count[256] = {0};
    for (int i = 0; i < N; ++i) count[sigma[i]] += 1;
    int best = 0;
    for (int k = 0; k < q; ++k)
        if (count[k] > best) best = count[k];
    return best;
}

/* Class of n_max among n_obins equal integer classes of [ceil(N/q), N]. */
int orc_obin(int n_max, int N, int q, int n_obins)
{
    int lo = (N + q - 1) / q;
    return (int)((int64_t)(n_max - lo) * n_obins / (N - lo + 1));
}

void orc_wl_steps(orc_rewl *s, int g, int64_t n)
{
    int N = s->N, q = s->q, L = s->L;
    int w = g / s->m;
    int32_t lo = s->e_lo[w], hi = lo + s->W;
    uint8_t *sg = s->sigma + (size_t)g * N;
    double *lg = s->lng + (size_t)g * (s->W + 1);
    uint32_t *Hg = s->H + (size_t)g * (s->W + 1);
    double lnf = s->lnf[w];
    int32_t E = s->E[g];
    uint64_t t = s->t[g];
    uint32_t r[4];
    for (int64_t i = 0; i < n; ++i, ++t) {
        orc_draw(s->seed, (uint32_t)t, (uint32_t)(t >> 32), (uint32_t)g, ORC_DOM_WL, r);
        int site = (int)orc_below(r[0], (uint32_t)N);
        int cur = sg[site];
        int v = (int)orc_below(r[1], (uint32_t)(q - 1));
        int nw = v + (v >= cur);
        int32_t En = E + orc_delta_e(L, sg, site, cur, nw);
        if (En >= lo && En <= hi) {
            double d = lg[E - lo] - lg[En - lo];
            if (orc_decide(s, 0, (uint64_t)g, t, d, orc_u53(r[2], r[3]))) {
                sg[site] = (uint8_t)nw;
                E = En;
            }
        }
        lg[E - lo] += lnf;
        Hg[E - lo] += 1u;
        if (s->production) {
            int o = orc_obin(orc_majority(sg, N, q), N, q, s->n_obins);
            s->heo[((size_t)w * (s->W + 1) + (size_t)(E - lo)) * s->n_obins + o] += 1u;
        }
    }
    s->E[g] = E;
    s->t[g] = t;
}

/* K steps for every walker of every window that has not finished. */
void orc_sweep(orc_rewl *s)
{
    for (int w = 0; w < s->h; ++w) {
        if (s->done[w]) continue;
        for (int k = 0; k < s->m; ++k) orc_wl_steps(s, w * s->m + k, s->K);
    }
}

/* ------------------------------------------------------------------------- */
/* Pairwise tree sum in index order (stride 1, 2, 4, ...; an element without a
 * partner passes through), then division by m: the mean of Sec. 2's merge. */
double orc_tree_mean(const double *v, int m)
{
    if (m < 1) return 0.0;
    double buf[4096];
    double *a = m <= 4096 ? buf : (double *)malloc(sizeof(double) * (size_t)m);
    for (int k = 0; k < m; ++k) a[k] = v[k];
    for (int stride = 1; stride < m; stride *= 2)
        for (int k = 0; k + stride < m; k += 2 * stride) a[k] = a[k] + a[k + stride];
    double mean = a[0] / (double)m;
    if (a != buf) free(a);
    return mean;
}

/* (a) Every bin any walker of the window has visited joins the window's mask. */
void orc_update_mask(orc_rewl *s)
{
    size_t B = (size_t)s->W + 1;
    for (int w = 0; w < s->h; ++w) {
        if (s->done[w]) continue;
        for (int k = 0; k < s->m; ++k) {
            const uint32_t *Hg = s->H + ((size_t)w * s->m + k) * B;
            for (size_t b = 0; b < B; ++b)
                if (Hg[b] > 0) s->mask[(size_t)w * B + b] = 1;
        }
    }
}

/* (b) Flatness of one walker over its window's mask: min H >= p * mean H
 * (each walker is judged on its own, Sec. 2). */
int orc_walker_flat(const orc_rewl *s, int g)
{
    size_t B = (size_t)s->W + 1;
    int w = g / s->m;
    const uint32_t *Hg = s->H + (size_t)g * B;
    const uint8_t *mk = s->mask + (size_t)w * B;
    uint64_t n = 0, sum = 0;
    uint32_t mn = UINT32_MAX;
    for (size_t b = 0; b < B; ++b) {
        if (!mk[b]) continue;
        n += 1;
        sum += Hg[b];
        if (Hg[b] < mn) mn = Hg[b];
    }
    if (n == 0) return 0;
    return (double)mn >= s->flatness * ((double)sum / (double)n);
}

/* Criterion of the first stage of the 1/t rule (Belardinelli & Pereyra,
 * Phys. Rev. E 75, 046701 (2007)): walker g has visited every bin of its
 * window's mask at least once since H was last cleared. */
int orc_walker_visited_all(const orc_rewl *s, int g)
{
    size_t B = (size_t)s->W + 1;
    int w = g / s->m;
    const uint32_t *Hg = s->H + (size_t)g * B;
    const uint8_t *mk = s->mask + (size_t)w * B;
    int n = 0;
    for (size_t b = 0; b < B; ++b) {
        if (!mk[b]) continue;
        n += 1;
        if (Hg[b] == 0) return 0;
    }
    return n > 0;
}

/* (c) A window whose m walkers are all flat averages and redistributes ln g,
 * clears H and moves to ln f / 2 (f -> sqrt f); it is finished once
 * ln f < ln f_final (Sec. 2).
 *
 * With the 1/t rule (schedule 1; Sec. 2 notes that the scheme works with any
 * valid WL update rule; the rule is Belardinelli & Pereyra's): the iteration
 * criterion is "every mask bin visited" instead of flatness; at the end of an
 * iteration ln f is halved unless the half falls below 1/t, where
 * t = (WL steps per walker) / (bins in the window's mask), and from then on the
 * window follows ln f = 1/t: at every barrier its walkers' ln g are merged,
 * H is cleared and ln f = 1/t is taken with the current t (held over the next
 * K steps).  Finished once ln f < ln f_final, as with halving. */
void orc_window_iterations(orc_rewl *s)
{
    size_t B = (size_t)s->W + 1;
    int m = s->m;
    double *col = (double *)malloc(sizeof(double) * (size_t)m);
    for (int w = 0; w < s->h; ++w) {
        if (s->done[w]) continue;
        int inv_t = s->schedule == 1;
        int follows_1t = inv_t && s->phase[w];
        if (!follows_1t) {
            int all_flat = 1;
            for (int k = 0; k < m; ++k)
                all_flat &= inv_t ? orc_walker_visited_all(s, w * m + k) : orc_walker_flat(s, w * m + k);
            if (!all_flat) continue;
        }
        for (size_t b = 0; b < B; ++b) {
            for (int k = 0; k < m; ++k) col[k] = s->lng[((size_t)w * m + k) * B + b];
            double mean = orc_tree_mean(col, m);
            for (int k = 0; k < m; ++k) s->lng[((size_t)w * m + k) * B + b] = mean;
        }
        for (int k = 0; k < m; ++k) memset(s->H + ((size_t)w * m + k) * B, 0, B * sizeof(uint32_t));
        if (!inv_t) {
            s->lnf[w] = s->lnf[w] * 0.5;
            s->iter[w] += 1;
        } else {
            int n_bins = 0;
            for (size_t b = 0; b < B; ++b) n_bins += s->mask[(size_t)w * B + b] != 0;
            uint64_t steps = s->t[(size_t)w * m];
            double one_over_t = steps ? (double)n_bins / (double)steps : 0.0;
            if (follows_1t) {
                s->lnf[w] = one_over_t;
            } else {
                double half = s->lnf[w] * 0.5;
                s->iter[w] += 1;
                if (half < one_over_t) {
                    s->phase[w] = 1;
                    s->lnf[w] = one_over_t;
                } else {
                    s->lnf[w] = half;
                }
            }
        }
        if (s->lnf[w] < s->lnf_final) s->done[w] = 1;
    }
    free(col);
}

void orc_set_schedule(orc_rewl *s, int schedule) { s->schedule = schedule; }

/* (d) Replica exchange between windows a and a+1 for every a with
 * a = round (mod 2) where neither window has finished.  Walker k of window a
 * is matched with walker pi(k) of window a+1 (pi: Fisher-Yates shuffle), and
 * the pair swaps configurations with probability Eq. 1. */
void orc_exchange(orc_rewl *s)
{
    int m = s->m, N = s->N;
    size_t B = (size_t)s->W + 1;
    uint32_t rnd = (uint32_t)s->round;
    int *pi = (int *)malloc(sizeof(int) * (size_t)m);
    uint8_t *tmp = (uint8_t *)malloc((size_t)N);
    uint32_t r[4];
    for (int a = (int)(s->round & 1); a + 1 < s->h; a += 2) {
        if (!s->production && (s->done[a] || s->done[a + 1])) continue;
        for (int k = 0; k < m; ++k) pi[k] = k;
        for (int i = m - 1; i >= 1; --i) {
            int n = m - 1 - i;
            orc_draw(s->seed, rnd, (uint32_t)(n >> 2), (uint32_t)a, ORC_DOM_PERM, r);
            int j = (int)orc_below(r[n & 3], (uint32_t)(i + 1));
            int tswap = pi[i]; pi[i] = pi[j]; pi[j] = tswap;
        }
        int32_t lo_a = s->e_lo[a], lo_b = s->e_lo[a + 1];
        int32_t hi_a = lo_a + s->W, hi_b = lo_b + s->W;
        for (int k = 0; k < m; ++k) {
            int gi = a * m + k, gj = (a + 1) * m + pi[k];
            int32_t Ei = s->E[gi], Ej = s->E[gj];
            if (!(Ei >= lo_b && Ei <= hi_b && Ej >= lo_a && Ej <= hi_a)) continue;
            const double *li = s->lng + (size_t)gi * B;
            const double *lj = s->lng + (size_t)gj * B;
            /* ln of Eq. 1's ratio; walker i carries X (energy Ei), j carries Y. */
            double d = (li[Ei - lo_a] - li[Ej - lo_a]) + (lj[Ej - lo_b] - lj[Ei - lo_b]);
            orc_draw(s->seed, rnd, (uint32_t)k, (uint32_t)a, ORC_DOM_XACC, r);
            s->xtried += 1;
            if (!orc_decide(s, 1, (uint64_t)gi, (uint64_t)s->round, d, orc_u53(r[0], r[1]))) continue;
            s->xacc += 1;
            memcpy(tmp, s->sigma + (size_t)gi * N, (size_t)N);
            memcpy(s->sigma + (size_t)gi * N, s->sigma + (size_t)gj * N, (size_t)N);
            memcpy(s->sigma + (size_t)gj * N, tmp, (size_t)N);
            s->E[gi] = Ej; s->E[gj] = Ei;
            uint32_t rr = s->rep[gi]; s->rep[gi] = s->rep[gj]; s->rep[gj] = rr;
        }
    }
    free(pi);
    free(tmp);
}

/* The barrier after every K steps: (a) mask, (b)+(c) flatness and window
 * iterations, (d) exchange, (e) next round. */
int orc_barrier(orc_rewl *s)
{
    size_t total = (size_t)s->h * s->m * ((size_t)s->W + 1);
    for (size_t i = 0; i < total; ++i)
        if (s->H[i] >= 0x80000000u) s->status = ORC_ERR_OVERFLOW;
    if (s->status) return s->status;
    orc_update_mask(s);
    orc_window_iterations(s);
    orc_exchange(s);
    orc_track_round_trips(s);
    s->round += 1;
    return ORC_OK;
}

int orc_all_done(const orc_rewl *s)
{
    for (int w = 0; w < s->h; ++w)
        if (!s->done[w]) return 0;
    return 1;
}

/* Rounds of (sweep, barrier) until every window is finished (Sec. 2) or
 * max_rounds rounds have run (max_rounds <= 0: no limit). */
int orc_run(orc_rewl *s, int64_t max_rounds, int *converged)
{
    int64_t n = 0;
    while (!orc_all_done(s) && (max_rounds <= 0 || n < max_rounds)) {
        if (s->round >= 0xffffffffll) return ORC_ERR_STATE;
        orc_sweep(s);
        int st = orc_barrier(s);
        if (st) return st;
        ++n;
    }
    if (converged) *converged = orc_all_done(s);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Fixed-weight production run.  After g(E) has been estimated, the paper goes
 * on sampling with the fixed weights 1/g(E) and measures distributions H(E,O)
 * of observables (Sec. 3.2, for the lipid model; here O is the Potts majority
 * count).  Every window keeps its walkers' ln g, and with ln f = 0 a WL step
 * is exactly a Metropolis step with weights 1/g(E) restricted to the window;
 * after each step H(E,O) of the window counts the walker's (E, class of O).
 * A production round: K such steps of every walker of every window (finished
 * or not), H cleared (it only counts the round's visits), replica exchange
 * (Eq. 1, which keeps detailed balance of the fixed-weight ensembles) between
 * every pair (a, a+1) with a = round (mod 2), round + 1.  No flatness check,
 * merge or f-reduction. */
int orc_production_start(orc_rewl *s, int n_obins)
{
    int lo = (s->N + s->q - 1) / s->q;
    if (n_obins < 1 || n_obins > s->N - lo + 1) return ORC_ERR_ARG;
    size_t n = (size_t)s->h * ((size_t)s->W + 1) * (size_t)n_obins;
    free(s->heo);
    s->heo = (uint64_t *)calloc(n, sizeof(uint64_t));
    if (!s->heo) return ORC_ERR_NOMEM;
    s->n_obins = n_obins;
    s->production = 1;
    for (int w = 0; w < s->h; ++w) s->lnf[w] = 0.0;
    memset(s->H, 0, sizeof(uint32_t) * (size_t)s->h * s->m * ((size_t)s->W + 1));
    return ORC_OK;
}

int orc_production_run(orc_rewl *s, int64_t rounds)
{
    if (!s->production) return ORC_ERR_STATE;
    for (int64_t r = 0; r < rounds; ++r) {
        for (int g = 0; g < s->h * s->m; ++g) orc_wl_steps(s, g, s->K);
        memset(s->H, 0, sizeof(uint32_t) * (size_t)s->h * s->m * ((size_t)s->W + 1));
        orc_exchange(s);
        orc_track_round_trips(s);
        s->round += 1;
    }
    return ORC_OK;
}

void orc_get_heo(const orc_rewl *s, uint64_t *o)
{
    if (s->heo) memcpy(o, s->heo, sizeof(uint64_t) * (size_t)s->h * ((size_t)s->W + 1) * (size_t)s->n_obins);
}

/* ------------------------------------------------------------------------- */
/* Joining the windows' pieces (Sec. 2, Fig. 2): for each neighbouring pair,
 * the joining bin is where beta = d ln g / dE of the two pieces agree best;
 * the upper piece is shifted to meet the lower one there, the lower piece is
 * used up to that bin and the upper one above it.  beta at bin b of a piece is
 * the difference quotient between the nearest masked bins on either side.
 * Input: per-window ln g (h x (W+1)) and masks.  Output: 2N+1 values, -inf for
 * bins no window visited.  Returns 0, or ORC_ERR_STATE if a pair has no
 * usable joining bin. */
static int orc_beta(const double *lg, const uint8_t *mk, int B, int i, double *beta)
{
    if (!mk[i]) return 0;
    int lo = i - 1, hi = i + 1;
    while (lo >= 0 && !mk[lo]) --lo;
    while (hi < B && !mk[hi]) ++hi;
    if (lo < 0 || hi >= B) return 0;
    *beta = (lg[hi] - lg[lo]) / (double)(hi - lo);
    return 1;
}

int orc_join_pieces(int N, int h, int W, const int32_t *e_lo, const double *lng_w,
                    const uint8_t *mask_w, double *out)
{
    int B = W + 1;
    int nb = 2 * N + 1;
    double *shift = (double *)calloc((size_t)h, sizeof(double));
    int *cut = (int *)malloc(sizeof(int) * (size_t)(h > 1 ? h - 1 : 1));
    int prev_cut = -1;
    for (int a = 0; a + 1 < h; ++a) {
        int ba = e_lo[a] + 2 * N, bb = e_lo[a + 1] + 2 * N;
        const double *la = lng_w + (size_t)a * B, *lb = lng_w + (size_t)(a + 1) * B;
        const uint8_t *ma = mask_w + (size_t)a * B, *mb = mask_w + (size_t)(a + 1) * B;
        int best = -1;
        double best_diff = 0.0;
        for (int b = bb; b <= ba + W; ++b) {
            if (b <= prev_cut) continue;
            double beta_a, beta_b;
            if (!orc_beta(la, ma, B, b - ba, &beta_a)) continue;
            if (!orc_beta(lb, mb, B, b - bb, &beta_b)) continue;
            double diff = fabs(beta_a - beta_b);
            if (best < 0 || diff < best_diff) {
                best = b;
                best_diff = diff;
            }
        }
        if (best < 0) {
            free(shift); free(cut);
            return ORC_ERR_STATE;
        }
        shift[a + 1] = (la[best - ba] + shift[a]) - lb[best - bb];
        cut[a] = best;
        prev_cut = best;
    }
    for (int b = 0; b < nb; ++b) out[b] = -INFINITY;
    for (int a = 0; a < h; ++a) {
        int base = e_lo[a] + 2 * N;
        int from = a == 0 ? base : cut[a - 1] + 1;
        int to = a == h - 1 ? base + W : cut[a];
        for (int b = from; b <= to; ++b)
            if (mask_w[(size_t)a * B + (b - base)]) out[b] = lng_w[(size_t)a * B + (b - base)] + shift[a];
    }
    free(shift); free(cut);
    return ORC_OK;
}

/* Normalisation: sum over visited bins of g = q^N, i.e. the log-sum-exp of ln g
 * equals N ln q (the total number of Potts configurations). */
void orc_normalise(int q, int N, double *lng, int nb)
{
    double mx = -INFINITY;
    for (int b = 0; b < nb; ++b)
        if (lng[b] > mx) mx = lng[b];
    if (mx == -INFINITY) return;
    double sum = 0.0;
    for (int b = 0; b < nb; ++b)
        if (lng[b] != -INFINITY) sum += exp(lng[b] - mx);
    double c = (double)N * log((double)q) - (mx + log(sum));
    for (int b = 0; b < nb; ++b)
        if (lng[b] != -INFINITY) lng[b] += c;
}

/* Joined, normalised ln g of a run (walker 0 of each window holds the merged
 * estimate once the window has finished). */
int orc_get_lng_joined(const orc_rewl *s, double *out)
{
    size_t B = (size_t)s->W + 1;
    double *lw = (double *)malloc(sizeof(double) * (size_t)s->h * B);
    for (int w = 0; w < s->h; ++w)
        memcpy(lw + (size_t)w * B, s->lng + (size_t)w * s->m * B, B * sizeof(double));
    int st = orc_join_pieces(s->N, s->h, s->W, s->e_lo, lw, s->mask, out);
    free(lw);
    if (st) return st;
    orc_normalise(s->q, s->N, out, 2 * s->N + 1);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Plain accessors used by the Python test harness. */
void orc_dims(const orc_rewl *s, int64_t out[8])
{
    out[0] = s->q; out[1] = s->L; out[2] = s->N; out[3] = s->h;
    out[4] = s->m; out[5] = s->W; out[6] = s->K; out[7] = s->round;
}
void orc_get_e_lo(const orc_rewl *s, int32_t *o) { memcpy(o, s->e_lo, sizeof(int32_t) * (size_t)s->h); }
void orc_get_sigma(const orc_rewl *s, uint8_t *o) { memcpy(o, s->sigma, (size_t)s->h * s->m * s->N); }
void orc_get_E(const orc_rewl *s, int32_t *o) { memcpy(o, s->E, sizeof(int32_t) * (size_t)s->h * s->m); }
void orc_get_rep(const orc_rewl *s, uint32_t *o) { memcpy(o, s->rep, sizeof(uint32_t) * (size_t)s->h * s->m); }
void orc_get_t(const orc_rewl *s, uint64_t *o) { memcpy(o, s->t, sizeof(uint64_t) * (size_t)s->h * s->m); }
void orc_get_lng(const orc_rewl *s, double *o)
{
    memcpy(o, s->lng, sizeof(double) * (size_t)s->h * s->m * ((size_t)s->W + 1));
}
void orc_get_H(const orc_rewl *s, uint32_t *o)
{
    memcpy(o, s->H, sizeof(uint32_t) * (size_t)s->h * s->m * ((size_t)s->W + 1));
}
void orc_get_mask(const orc_rewl *s, uint8_t *o) { memcpy(o, s->mask, (size_t)s->h * ((size_t)s->W + 1)); }
void orc_get_lnf(const orc_rewl *s, double *o) { memcpy(o, s->lnf, sizeof(double) * (size_t)s->h); }
void orc_get_iter(const orc_rewl *s, int32_t *o) { memcpy(o, s->iter, sizeof(int32_t) * (size_t)s->h); }
void orc_get_done(const orc_rewl *s, uint8_t *o) { memcpy(o, s->done, (size_t)s->h); }
void orc_get_xstats(const orc_rewl *s, uint64_t o[2]) { o[0] = s->xtried; o[1] = s->xacc; }
void orc_get_rt_end(const orc_rewl *s, uint8_t *o) { memcpy(o, s->rt_end, (size_t)s->h * s->m); }
void orc_get_phase(const orc_rewl *s, uint8_t *o) { memcpy(o, s->phase, (size_t)s->h); }
void orc_get_rt_trips(const orc_rewl *s, uint32_t *o)
{
    memcpy(o, s->rt_trips, sizeof(uint32_t) * (size_t)s->h * s->m);
}

void orc_set_lng(orc_rewl *s, const double *v)
{
    memcpy(s->lng, v, sizeof(double) * (size_t)s->h * s->m * ((size_t)s->W + 1));
}
void orc_set_lnf(orc_rewl *s, const double *v) { memcpy(s->lnf, v, sizeof(double) * (size_t)s->h); }
void orc_set_H(orc_rewl *s, const uint32_t *v)
{
    memcpy(s->H, v, sizeof(uint32_t) * (size_t)s->h * s->m * ((size_t)s->W + 1));
}
void orc_set_mask(orc_rewl *s, const uint8_t *v) { memcpy(s->mask, v, (size_t)s->h * ((size_t)s->W + 1)); }
/* Give walker g a configuration; its energy is recounted. */
void orc_set_config(orc_rewl *s, int g, const uint8_t *sigma)
{
    memcpy(s->sigma + (size_t)g * s->N, sigma, (size_t)s->N);
    s->E[g] = orc_energy(s->L, s->sigma + (size_t)g * s->N);
}
void orc_set_round(orc_rewl *s, int64_t r) { s->round = r; }
