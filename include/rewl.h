/*
 * rewl.h -- C ABI of the GB300 (sm_103a) implementation of Replica-Exchange
 * Wang-Landau sampling (REWL) for the periodic 2D q-state Potts model.
 *
 * Method: Vogel, Li, Wuest & Landau, "Exploring new frontiers in statistical
 * physics with a new, parallel Wang-Landau framework", arXiv:1312.3004.
 *   Sec. 2   -- the REWL scheme: the energy range is split into h windows with
 *               overlap o; every window is sampled by m independent WL walkers
 *               with their own ln g(E) and H(E); walkers accept single moves
 *               with min[1, g(E_old)/g(E_new)] and add ln f to ln g(E) and 1 to
 *               H(E) every step; once all m walkers of a window are flat their
 *               ln g are averaged and shared, H is cleared and f -> sqrt(f);
 *               configurations are exchanged between walkers of neighbouring
 *               windows with the probability of Eq. 1; the run ends when every
 *               window has reached f_final and the pieces are joined where
 *               their slopes d ln g / dE agree best (Fig. 2).
 *   Eq. 2    -- Potts energy E = -sum over nearest-neighbour pairs of
 *               delta(s_i, s_j); N = L x L spins, periodic here.
 *
 * Conventions for every function below:
 *   - Every call returns a rewl_status; nothing throws across the ABI.  On an
 *     error, rewl_last_error() returns a message (thread-local, valid until the
 *     next call on the same thread).
 *   - A rewl_t handle owns all device memory of one REWL instance.  It lives on
 *     the CUDA device that was current when it was created.
 *   - Output buffers are owned by the caller.  "host" buffers must be host
 *     memory (pageable or pinned); no function keeps a pointer to them.
 *   - Calls on one handle are not thread-safe; distinct handles are
 *     independent.  Work is queued on the handle's stream (see
 *     rewl_set_stream); functions that return results to host memory
 *     synchronise that stream.
 *   - Energies use E in [-2N, 0]; bin index b = E + 2N in [0, 2N] is the number
 *     of unsatisfied bonds.  Window i covers E_lo(i) .. E_lo(i) + W (W + 1 bins)
 *     with W = ceil(2N / (1 + (h - 1)(1 - o))) and
 *     E_lo(i) = -2N + round_half_up(i (2N - W) / (h - 1)).
 */
#ifndef REWL_H
#define REWL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rewl_s *rewl_t;

typedef enum {
    REWL_OK = 0,
    REWL_ERR_ARG = 1,       /* an argument is out of range or a pointer is NULL   */
    REWL_ERR_NOMEM = 2,     /* a device or host allocation failed                 */
    REWL_ERR_CUDA = 3,      /* a CUDA runtime call failed                          */
    REWL_ERR_TIMEOUT = 4,   /* the stall watchdog gave up (REWL_OPT_STALL_MS)      */
    REWL_ERR_OVERFLOW = 5,  /* a histogram bin reached 2^31 visits                 */
    REWL_ERR_STATE = 6,     /* call not valid in the current state (see function) */
    REWL_ERR_CANCELLED = 7  /* the job was cancelled                               */
} rewl_status;

/* Parameters of one REWL instance (Sec. 2 symbols). */
typedef struct rewl_params {
    int q;                        /* Potts states, 2 <= q <= 255 (<= 16 for 4-bit spins) */
    int L;                        /* linear size, 3 <= L <= 1024; N = L * L               */
    int h;                        /* number of energy windows, >= 1                        */
    double overlap;               /* o, 0 <= o < 1 (0.75 in the paper)                     */
    int m;                        /* walkers per window, 1 <= m <= 256                     */
    double lnf_final;             /* stop once ln f < lnf_final, 0 < lnf_final < 1         */
    double flatness;              /* p: flat iff min H >= p * mean H, 0 < p < 1            */
    long long exchange_interval;  /* K: WL steps per walker between exchanges, >= 1       */
    unsigned long long seed;      /* Philox4x32-10 key                                     */
} rewl_params;

/* Derived sizes of an instance, filled by rewl_get_info. */
typedef struct rewl_info {
    int N;              /* spins per configuration                          */
    int W;              /* window width in energy units (W + 1 bins)         */
    int walkers;        /* h * m                                             */
    int spin_bits;      /* 4 or 8 bits per stored spin                       */
    size_t device_bytes;/* device memory owned by the handle                 */
} rewl_info;

/* Per-instance counters, filled by rewl_get_stats. */
typedef struct rewl_stats {
    long long rounds;          /* exchange rounds completed (barriers)         */
    long long flips;           /* WL proposals made by all walkers             */
    long long accepted;        /* accepted WL proposals                        */
    long long exch_tried;      /* exchange pairs evaluated with Eq. 1          */
    long long exch_accepted;   /* exchanges carried out                        */
    long long near_ties;       /* acceptance draws with |u - exp(D)| < 1e-14   */
    long long slow_decisions;  /* WL decisions the fast sweep took in binary64 */
    long long seq_steps;       /* WL steps the fast sweep resolved one at a time */
    int windows_done;          /* windows that reached ln f_final              */
    int converged;             /* 1 when every window is done                  */
    double min_lnf;            /* smallest ln f over windows                   */
    double max_lnf;            /* largest ln f over windows                    */
} rewl_stats;

/* Create an instance: computes the window table, allocates the device state,
 * draws every walker's initial configuration from the seed and moves it into
 * its window (Sec. 3.2: each walker starts with a configuration whose energy is
 * inside its window).  ln g = 0, H = 0 and ln f = 1 in every window.
 * Arguments as in rewl_params.  *out receives the handle (NULL on error).
 * Errors: REWL_ERR_ARG (a parameter out of range, W < 8 bins, or a lattice too
 * large for one CTA's shared memory), REWL_ERR_NOMEM, REWL_ERR_CUDA,
 * REWL_ERR_STATE (a walker could not reach its window within the bounded
 * number of entry moves). */
rewl_status rewl_create(int q, int L, int h, double overlap, int m, double lnf_final,
                        double flatness, long long exchange_interval,
                        unsigned long long seed, rewl_t *out);

/* As rewl_create, from a parameter struct.  spin_bits: 0 picks 4 bits when
 * q <= 16 and 8 bits otherwise; 4 or 8 force the packing. */
rewl_status rewl_create_ext(const rewl_params *params, int spin_bits, rewl_t *out);

/* Queue subsequent work of the handle on `stream` (a cudaStream_t passed as
 * void*; NULL selects the handle's own stream).  Runtime plumbing with no
 * counterpart in the paper.  The stream must belong to the
 * handle's device and outlive its use by the handle. */
rewl_status rewl_set_stream(rewl_t h, void *stream);

/* Run exchange rounds (Sec. 2): each round is K WL steps of every walker of
 * every unfinished window, then the barrier: visited-bin mask, flatness of
 * every walker, merge + f-reduction of flat windows, replica exchange (Eq. 1)
 * between windows (a, a+1) with a = round mod 2.  Runs until every window has
 * ln f < lnf_final, or until max_rounds rounds have been queued
 * (max_rounds <= 0: no limit).  Rounds after convergence change nothing.
 * Synchronises the stream; *converged (may be NULL) is 1 once every window is
 * done.  Errors: REWL_ERR_OVERFLOW, REWL_ERR_CUDA, REWL_ERR_ARG. */
rewl_status rewl_run(rewl_t h, long long max_rounds, int *converged);

/* Queue exactly `rounds` exchange rounds (Sec. 2, as rewl_run) on the handle's
 * stream and return without synchronising (for timing with events on that
 * stream).  Status
 * flags are checked by the next synchronising call. */
rewl_status rewl_run_async(rewl_t h, long long rounds);

/* Queue one phase of an exchange round (Sec. 2) on the handle's stream without
 * synchronising: REWL_PHASE_SWEEP (K WL steps of every walker of every
 * unfinished window), REWL_PHASE_CHECK (mask, flatness, merge, f-reduction),
 * REWL_PHASE_EXCHANGE (replica exchange, then round + 1).  A round is the
 * three phases in this order; queuing them one by one lets a caller put
 * timing events between them.  Errors: REWL_ERR_ARG (unknown phase),
 * REWL_ERR_CUDA (launch failure). */
enum { REWL_PHASE_SWEEP = 0, REWL_PHASE_CHECK = 1, REWL_PHASE_EXCHANGE = 2 };
rewl_status rewl_run_phase(rewl_t h, int phase);

/* Options of a handle.  All but REWL_OPT_SCHEDULE are tuning options (no
 * counterpart in the paper, and no effect on results: every choice computes
 * the same states bit for bit):
 *   REWL_OPT_SWEEP_KERNEL  0 = fast sweep (integer acceptance path with a
 *                          binary64 fallback), 1 = binary64 reference sweep
 *   REWL_OPT_LANES         lanes per walker of the fast sweep: 0 = chosen from
 *                          the walker count and lattice size (up to 80 walkers
 *                          per SM 32, or 8 for lattices of at most 128 sites;
 *                          else 1; and 1 whenever a lane group's ln g shadow
 *                          would not fit in shared memory), or
 *                          1, 2, 4, 8, 16, 32
 *   REWL_OPT_WALKERS_PER_CTA  (read-only) walkers per CTA of the current plan
 *   REWL_OPT_LATTICE       where the fast sweep keeps the lattices: set 0 =
 *                          chosen (global memory above 16 KB each, and with
 *                          one lane per walker; else shared memory), 1 =
 *                          global memory (L2), 2 = shared memory; with one
 *                          lane per walker, global means the walker's whole
 *                          state (its ln g shadow too) stays in global memory;
 *                          get: 1 if the current plan keeps them in global
 *                          memory, else 0
 *   REWL_OPT_STALL_MS      stall watchdog of rewl_run: when no window has
 *                          finished an iteration (or follows ln f = 1/t, which
 *                          falls every round) for this many milliseconds
 *                          of the call, rewl_run stops at a round boundary
 *                          and returns REWL_ERR_TIMEOUT (the state stays valid
 *                          and the run can go on); 0 (default) = off
 *   REWL_OPT_SCHEDULE      the ln f schedule of every window (Sec. 2 states that
 *                          the scheme works with any valid WL update rule):
 *                          0 (default) = ln f / 2 once all m walkers are flat
 *                          (Sec. 2); 1 = the 1/t rule of Belardinelli & Pereyra
 *                          (Phys. Rev. E 75, 046701): an iteration ends once every
 *                          walker has visited every bin of the window's mask
 *                          (flatness is not used), ln f is halved unless the
 *                          half is below 1/t with t = WL steps per walker / bins
 *                          in the mask, and from then on (REWL_FIELD_PHASE = 1)
 *                          every barrier merges the window's walkers, clears H
 *                          and sets ln f = 1/t; done once ln f < lnf_final.  Set
 *                          it at a round boundary; rounds run before keep their
 *                          schedule.  Not available on batch instances.
 * rewl_set_option synchronises the stream and re-plans the sweep (not for
 * REWL_OPT_STALL_MS).
 * Errors: REWL_ERR_ARG (unknown option or value, or a plan that does not fit
 * in shared memory). */
enum {
    REWL_OPT_SWEEP_KERNEL = 0, REWL_OPT_LANES = 1, REWL_OPT_WALKERS_PER_CTA = 2, REWL_OPT_LATTICE = 3,
    REWL_OPT_STALL_MS = 4, REWL_OPT_SCHEDULE = 5
};
rewl_status rewl_set_option(rewl_t h, int option, long long value);
rewl_status rewl_get_option(rewl_t h, int option, long long *value);

/* Synchronise the handle's stream and report its device status:
 * *converged (may be NULL) as in rewl_run (Sec. 2's global termination: every
 * window below f_final).  Errors: REWL_ERR_OVERFLOW, REWL_ERR_CUDA. */
rewl_status rewl_sync(rewl_t h, int *converged);

/* The joined, normalised ln g over all 2N + 1 bins (Sec. 2, Fig. 2): for each
 * pair of neighbouring windows the joining bin is the one where the
 * central-difference slopes of the two pieces agree best; the upper piece is
 * shifted to meet the lower one there.  Normalised so that sum_E g(E) = q^N.
 * out: caller-owned host array of len = 2N + 1 doubles; out[b] = ln g(E = b - 2N),
 * -INFINITY for bins no walker visited.  partial = 0 requires a converged run
 * (else REWL_ERR_STATE); partial = 1 joins the current estimates. */
rewl_status rewl_get_lng(rewl_t h, double *out, size_t len, int partial);

/* ln g of window w as held by its walker 0 (W + 1 doubles into `out`, host),
 * and the window's lowest energy in *e_lo (may be NULL).  After a merge every
 * walker of the window holds the same average (Sec. 2), so walker 0 stands for
 * the window; unjoined and unnormalised (Fig. 2 before the join).
 * Errors: REWL_ERR_ARG (w outside [0, h), len != W + 1). */
rewl_status rewl_get_window_lng(rewl_t h, int w, double *out, size_t len, int *e_lo);

/* Sizes of the instance (W from the window formula of Sec. 2 / Fig. 1). */
rewl_status rewl_get_info(rewl_t h, rewl_info *info);

/* Counters of the instance (synchronises the stream): WL proposals and
 * acceptances (Sec. 2's single-spin-flip steps, Sec. 3.1), Eq. 1 exchange
 * trials and acceptances, windows done; the fast-sweep counters describe the
 * implementation, not the method. */
rewl_status rewl_get_stats(rewl_t h, rewl_stats *stats);

/* Copy one state array of the instance to host memory (synchronises).  The
 * arrays are Sec. 2's per-walker state (configuration, E, ln g(E), H(E)) and
 * per-window state (ln f, iterations); the replica ids and round-trip counters
 * follow the replica paths through the windows that Fig. 7 plots:
 *   REWL_FIELD_SPINS  uint8  [h*m][N]  configuration held by walker g = i*m + k
 *   REWL_FIELD_ENERGY int32  [h*m]     its energy
 *   REWL_FIELD_REPLICA uint32 [h*m]    its replica id (initially g)
 *   REWL_FIELD_STEPS  uint64 [h*m]     WL steps made by walker g
 *   REWL_FIELD_LNG    double [h*m][W+1] ln g of walker g
 *   REWL_FIELD_HIST   uint32 [h*m][W+1] H of walker g in the current iteration
 *   REWL_FIELD_MASK   uint8  [h][W+1]  bins visited by any walker of window i
 *   REWL_FIELD_LNF    double [h]       ln f of window i
 *   REWL_FIELD_ITER   int32  [h]       completed iterations of window i
 *   REWL_FIELD_DONE   uint8  [h]       1 once ln f < lnf_final
 *   REWL_FIELD_ELO    int32  [h]       lowest energy of window i
 *   REWL_FIELD_ROUND  int64  [1]       exchange rounds completed
 *   REWL_FIELD_TRIPS  uint32 [h*m]     by replica id c: round trips completed, i.e.
 *                                      arrivals in window 0 after a visit to window
 *                                      h-1 since the last stay in window 0 (checked
 *                                      after each exchange round; 0 when h = 1)
 *   REWL_FIELD_TRIP_END uint8 [h*m]    by replica id c: last end of the range its
 *                                      window touched: 0 none yet, 1 window 0,
 *                                      2 window h-1
 *   REWL_FIELD_PHASE  uint8  [h]       1/t rule (REWL_OPT_SCHEDULE = 1): 1 once window i
 *                                      follows ln f = 1/t, else 0
 *   REWL_FIELD_TIES   uint64 [32][2]   the first 32 near-tie acceptance draws
 *                                      (|u - exp(D)| < 1e-14, where the exp of two
 *                                      libraries may decide differently; all of
 *                                      them are counted in rewl_stats.near_ties):
 *                                      entry i = (kind << 32 | who, when); kind 0 a
 *                                      WL step of walker slot `who` at its step
 *                                      index `when`; kind 1 an exchange of the pair
 *                                      whose lower-window walker is slot `who`, in
 *                                      round `when`; entries at or beyond
 *                                      near_ties are zero (read-only)
 * bytes must equal the size above, else REWL_ERR_ARG. */
enum {
    REWL_FIELD_SPINS = 0, REWL_FIELD_ENERGY = 1, REWL_FIELD_REPLICA = 2, REWL_FIELD_STEPS = 3,
    REWL_FIELD_LNG = 4, REWL_FIELD_HIST = 5, REWL_FIELD_MASK = 6, REWL_FIELD_LNF = 7,
    REWL_FIELD_ITER = 8, REWL_FIELD_DONE = 9, REWL_FIELD_ELO = 10, REWL_FIELD_ROUND = 11,
    REWL_FIELD_TRIPS = 12, REWL_FIELD_TRIP_END = 13, REWL_FIELD_PHASE = 14, REWL_FIELD_TIES = 15
};
rewl_status rewl_get_field(rewl_t h, int field, void *out, size_t bytes);

/* Overwrite one state array from host memory (same layouts as rewl_get_field;
 * REWL_FIELD_SPINS also recounts the energies; REWL_FIELD_ELO,
 * REWL_FIELD_REPLICA, REWL_FIELD_ENERGY and REWL_FIELD_TIES are read-only).
 * For tests that start from a chosen state, e.g. fixed weights with
 * ln f = 0. */
rewl_status rewl_set_field(rewl_t h, int field, const void *in, size_t bytes);

/* ---- Fixed-weight production (Sec. 3.2) -------------------------------------
 * After the density of states is estimated, the paper samples configurations
 * with the fixed weights 1/g(E) and records distributions H(E, O) of
 * observables.  For the Potts model the observable here is the majority count
 * O = max_v #{i : s_i = v} in [ceil(N/q), N], kept in n_obins equal integer
 * classes: class = (O - ceil(N/q)) * n_obins / (N - ceil(N/q) + 1).
 *
 * rewl_production_start: from the handle's current state (usually a converged
 * run) every window keeps its walkers' own ln g and sets ln f = 0 (a WL step
 * is then a Metropolis step with weights 1/g(E) inside the window), H is
 * cleared and the histogram H(E, O) of every window is zeroed.  Allocates the
 * histogram (h * (W + 1) * n_obins * 8 bytes) and spin counts (h * m * q * 4
 * bytes) through the allocator hook.  May be called again to restart the
 * histogram.  From then on rewl_run, rewl_run_async, rewl_run_phase,
 * rewl_set_option, rewl_save and rewl_load return REWL_ERR_STATE.
 * Errors: REWL_ERR_ARG (n_obins outside [1, N - ceil(N/q) + 1]),
 * REWL_ERR_NOMEM, REWL_ERR_CUDA, REWL_ERR_STATE (instance of a batch).
 *
 * rewl_production_run: `rounds` production rounds, each K steps of every
 * walker of every window (finished or not), each step followed by
 * H(E, class) += 1 in its window's histogram, then a replica exchange with
 * Eq. 1 between every pair (a, a + 1), a = round (mod 2), and round + 1.
 * Synchronises the handle's stream.  Errors: REWL_ERR_STATE (not started),
 * REWL_ERR_ARG (rounds < 0), REWL_ERR_CUDA.
 *
 * rewl_production_histogram: out[(w * (W + 1) + (E - E_lo(w))) * n_obins + class]
 * = visits of window w (caller-owned host buffer, len = h * (W + 1) *
 * n_obins), counted since rewl_production_start.  Errors: REWL_ERR_STATE
 * (not started), REWL_ERR_ARG (len). */
rewl_status rewl_production_start(rewl_t h, int n_obins);
rewl_status rewl_production_run(rewl_t h, long long rounds);
rewl_status rewl_production_histogram(rewl_t h, unsigned long long *out, size_t len);

/* Checkpoint and resume (no counterpart in the paper).
 * Serialise the whole state (at a round boundary) into `buf` (host).  With
 * buf == NULL only *len is set to the required size.  rewl_load restores it
 * into a handle created with the same parameters and set to the same ln f
 * schedule; run(2K) equals run(K) + save + load + run(K) bit for bit.
 * Errors: REWL_ERR_ARG (buffer too small, or a blob of other parameters or
 * schedule / corrupted). */
rewl_status rewl_save(rewl_t h, void *buf, size_t *len);
rewl_status rewl_load(rewl_t h, const void *buf, size_t len);

/* ---- Batches: many independent instances advanced together -----------------
 * A batch holds n instances of uneven (q, L, h, m) in one device allocation.
 * Each round runs one sweep launch per spin packing -- a persistent launch
 * that takes walker groups of every unfinished instance from a device queue
 * (lane groups), or one thread per walker of every instance (see
 * rewl_batch_create_ext) -- then one batched check launch
 * (every window of every instance) and one batched exchange launch; rounds
 * are replayed as a CUDA graph.  Every instance computes exactly the states it
 * computes alone (same parameters, same seed): batching changes the runtime,
 * not the arithmetic.  (Sec. 2's walkers and windows are independent between
 * barriers; instances are independent altogether.) */
typedef struct rewl_batch_s *rewl_batch_t;

/* Create a batch of n instances (jobs[i] as in rewl_create; spin_bits as in
 * rewl_create_ext, applied to all).  Errors as rewl_create, naming the job. */
rewl_status rewl_batch_create(const rewl_params *jobs, int n, int spin_bits, rewl_batch_t *out);
/* As rewl_batch_create, choosing how walkers map to threads: lanes = 32, a
 * group of 32 lanes per walker with its state staged in shared memory (walker
 * groups of one instance per CTA); lanes = 1, a thread per walker with all its
 * state in global memory (walkers of any instances in a CTA); lanes = 0,
 * chosen from the total walker count (1 from 16384 walkers on).  With one lane
 * and spin_bits = 0 the spins are packed 8 bits each.  Results are the same
 * either way.  Errors: REWL_ERR_ARG for another lanes value. */
rewl_status rewl_batch_create_ext(const rewl_params *jobs, int n, int spin_bits, int lanes, rewl_batch_t *out);

/* Autotuner (no counterpart in the paper: it picks how the batch runs, not
 * what it computes).  Times the batch's candidate configurations -- spin
 * packing 4 or 8 bits (when spin_bits was 0 and every q <= 16), walkers as lane
 * groups of 32 with 36, 72 or 110 KB of shared memory per sweep CTA (when
 * lanes was 0 and the walkers fit) or as a thread each with 128 or 256
 * threads per CTA -- each over `rounds` rounds (after one round that settles
 * it), by CUDA events on the batch's stream and the WL proposals counted, and
 * leaves the batch in the fastest one.  The rounds it runs are ordinary rounds
 * of every instance (no configuration changes a result).  The choice is
 * cached per batch signature (device, freedoms, every instance's q, L, h, m,
 * K) for the process: with rounds <= 0 a cached choice is applied without
 * timing (*from_cache = 1), else 2 rounds per candidate are timed.
 * entries[0 .. *n_entries - 1] (may be NULL with max_entries = 0) receive the
 * timed candidates.  Errors: REWL_ERR_ARG, REWL_ERR_NOMEM, REWL_ERR_CUDA. */
typedef struct rewl_tune_entry {
    int spin_bits;      /* 4 or 8 */
    int lanes;          /* 32 (lane groups) or 1 (a thread per walker) */
    int cta_kb;         /* lane groups: shared memory per sweep CTA (KB), else 0 */
    int threads;        /* a thread per walker: threads per CTA, else 0 */
    double flips_per_s; /* WL proposals per second measured */
} rewl_tune_entry;
rewl_status rewl_batch_autotune(rewl_batch_t b, int rounds, rewl_tune_entry *entries, int max_entries,
                                int *n_entries, int *from_cache);
/* The same for one handle (no counterpart in the paper): the fast sweep's lanes
 * per walker (32, 16, 8, 4, 2, 1; the lattice placed by the size rule) are
 * each timed over `rounds` rounds (<= 0: 2) after one settling round, and the
 * fastest is kept (REWL_OPT_LANES).  The rounds are ordinary rounds of the run:
 * the handle advances by (1 + rounds) rounds per candidate, and no choice
 * changes a result.  entries receive the timed candidates (spin_bits, lanes,
 * cta_kb = shared memory per CTA in KB, threads per CTA, flips_per_s).  Stops
 * early once the run has converged.  Errors: REWL_ERR_ARG, REWL_ERR_STATE
 * (instance of a batch, or in production), REWL_ERR_CUDA. */
rewl_status rewl_autotune(rewl_t h, int rounds, rewl_tune_entry *entries, int max_entries, int *n_entries);
/* The batch's current configuration (each pointer may be NULL; cta_kb is 0 for
 * a thread per walker, threads 0 for lane groups). */
rewl_status rewl_batch_config(rewl_batch_t b, int *spin_bits, int *lanes, int *cta_kb, int *threads);

/* Run rounds of every unfinished instance until all have converged or
 * max_rounds rounds were queued (<= 0: no limit); synchronises.
 * *n_converged (may be NULL) = instances whose windows are all done. */
rewl_status rewl_batch_run(rewl_batch_t b, long long max_rounds, int *n_converged);
/* Queue `rounds` rounds without synchronising / read the status. */
rewl_status rewl_batch_run_async(rewl_batch_t b, long long rounds);
rewl_status rewl_batch_sync(rewl_batch_t b, int *n_converged);
/* Stream for subsequent work (cudaStream_t as void*, NULL = own stream). */
rewl_status rewl_batch_set_stream(rewl_batch_t b, void *stream);

/* A read-only handle of instance i, owned by the batch: rewl_get_lng,
 * rewl_get_window_lng, rewl_get_field, rewl_set_field, rewl_get_info,
 * rewl_get_stats, rewl_save and rewl_load work on it; the functions that run
 * rounds, change options or streams return REWL_ERR_STATE; rewl_destroy on it
 * does nothing.  Valid until rewl_batch_destroy. */
rewl_status rewl_batch_instance(rewl_batch_t b, int i, rewl_t *view);

/* Sizes of a batch (each pointer may be NULL). */
rewl_status rewl_batch_info(rewl_batch_t b, int *n_instances, long long *walkers, size_t *device_bytes);

/* Counters summed over the instances (rounds = the largest round count;
 * windows_done = converged instances; converged = all instances done). */
rewl_status rewl_batch_stats(rewl_batch_t b, rewl_stats *stats);

/* Release a batch and all of its instances.  NULL is ignored. */
void rewl_batch_destroy(rewl_batch_t b);

/* ---- Serving: continuous batching of density-of-states jobs -----------------
 * A server owns a device memory pool of pool_bytes and at most max_jobs
 * resident jobs.  Submitted jobs wait in a first-come queue until their state
 * fits into the pool (admission by device footprint; a later, smaller job may
 * be admitted before an earlier one that does not fit yet).  Each
 * rewl_server_step admits what fits, advances every resident job by `rounds`
 * exchange rounds together (the batched kernels), and retires converged jobs:
 * their windows are joined on the host (Fig. 2 of the paper), the normalised
 * ln g is kept by the server, and their memory returns to the pool.  A job
 * computes exactly the states it computes when run alone.  Calls on one server
 * are not thread-safe. */
typedef struct rewl_server_s *rewl_server_t;
enum { REWL_JOB_QUEUED = 0, REWL_JOB_RUNNING = 1, REWL_JOB_DONE = 2, REWL_JOB_FAILED = 3, REWL_JOB_CANCELLED = 4 };

/* Errors: REWL_ERR_ARG (pool_bytes < 4096 or max_jobs < 1), REWL_ERR_NOMEM. */
rewl_status rewl_server_create(size_t pool_bytes, int max_jobs, rewl_server_t *out);
/* Queue a job (parameters as rewl_create_ext).  *job_id (may be NULL) names it.
 * Errors: REWL_ERR_ARG (parameters), REWL_ERR_NOMEM (larger than the pool). */
rewl_status rewl_server_submit(rewl_server_t s, const rewl_params *params, int spin_bits, long long *job_id);
/* Admit, advance every resident job by rounds (>= 1) rounds, retire; then
 * *n_running / *n_queued (may be NULL) count resident and waiting jobs.
 * The resident walkers run as lane groups of 32 (state staged in shared
 * memory) or a thread each (state in global memory): from 512 resident walkers
 * on, whenever their number has changed by half since the last choice, the
 * first two rounds of a step time one mapping each (CUDA events) and the faster
 * is kept (no counterpart in the paper; both compute the same states). */
rewl_status rewl_server_step(rewl_server_t s, long long rounds, int *n_running, int *n_queued);
/* The current mapping (*lanes = 32 or 1) and the resident walker count it was
 * chosen at (0: not timed, fewer than 512 walkers).  Each pointer may be NULL. */
rewl_status rewl_server_mapping(rewl_server_t s, int *lanes, long long *tuned_walkers);
/* *state = REWL_JOB_*. */
rewl_status rewl_server_poll(rewl_server_t s, long long job_id, int *state);
/* Joined, normalised ln g of a finished job into `out` (host, 2N + 1 doubles,
 * as rewl_get_lng).  Errors: REWL_ERR_STATE (not finished), REWL_ERR_CANCELLED,
 * the job's own error if it failed, REWL_ERR_ARG (unknown job, wrong len). */
rewl_status rewl_server_result(rewl_server_t s, long long job_id, double *out, size_t len);
/* times (may be NULL): [submitted, admitted, finished] in seconds of a steady
 * host clock; counts (may be NULL): [rounds, WL proposals, device bytes]. */
rewl_status rewl_server_job_info(rewl_server_t s, long long job_id, double *times, long long *counts);
/* Cancel a queued or running job (its memory returns to the pool). */
rewl_status rewl_server_cancel(rewl_server_t s, long long job_id);
/* Forget a finished, failed or cancelled job: its record and kept result are
 * freed, and the id becomes unknown (a long-running server calls this once it
 * has read a result).  Errors: REWL_ERR_ARG (unknown job), REWL_ERR_STATE (the
 * job is queued or running). */
rewl_status rewl_server_release(rewl_server_t s, long long job_id);
/* counts (may be NULL): [queued, running, done, failed or cancelled, rounds
 * stepped, WL proposals] (done / failed / cancelled: jobs not yet released);
 * *pool_free (may be NULL): free pool bytes. */
rewl_status rewl_server_info(rewl_server_t s, long long *counts, size_t *pool_free);
/* Release the server, its pool and every job.  NULL is ignored. */
void rewl_server_destroy(rewl_server_t s);

/* A whole run without allocating: for callers that cannot call cudaMalloc,
 * e.g. code under a framework whose caching allocator owns the device memory,
 * a process with a fixed device-memory budget, or a latency-critical loop that
 * cannot take the device-wide synchronisation of cudaMalloc / cudaFree.
 * (The paper has no counterpart: this is a deployment variant of
 * rewl_create + rewl_run.)
 *
 * Runs the instance described by `params` (spin_bits as in rewl_create_ext)
 * for up to max_rounds exchange rounds (<= 0: until converged) with all of its
 * working state in one fixed device array of 16 MiB that the library reserves
 * on every GPU that loads it, for the life of the process.  Calls no
 * cudaMalloc, cudaFree or other allocating routine.
 * Outputs (caller-owned DEVICE memory on the current device):
 *   lng_out  h * (W + 1) doubles: ln g of walker 0 of every window, window-major
 *            (the rows rewl_get_field(REWL_FIELD_LNG) holds for walkers i*m);
 *   mask_out h * (W + 1) bytes: visited-bin masks, or NULL;
 *   out_bins must equal h * (W + 1).
 * *converged (host, may be NULL) is 1 when every window finished.  Work is
 * queued on `stream` (cudaStream_t as void*, NULL = default stream) and the
 * call synchronises it before returning.
 * The first call on a device (and the first after that device's context was
 * reset) looks up the array's device address, with that device current, and
 * caches it for that context; make that first call before any stream capture.  The array is shared by every call: each call clears what must
 * start at zero, and calls whose work overlaps on the GPU race on it.
 * Errors: REWL_ERR_ARG (parameters, NULL lng_out, wrong out_bins, or an
 * instance whose state exceeds the 16 MiB array), REWL_ERR_CUDA,
 * REWL_ERR_OVERFLOW, REWL_ERR_STATE (window entry failed). */
rewl_status rewl_run_static(const rewl_params *params, int spin_bits, long long max_rounds,
                            double *lng_out, unsigned char *mask_out, size_t out_bins,
                            int *converged, void *stream);

/* Release the handle and its device memory.  NULL is ignored. */
void rewl_destroy(rewl_t h);

/* ---- Analysis of a density of states (host functions, no device work) -------
 * Each takes a joined ln g as rewl_get_lng returns it: lng[b] = ln g(E) for
 * E = b - 2N, b = 0 .. 2N (len = 2N + 1, so N = (len - 1) / 2), -INFINITY for
 * energies without configurations; NaN or +inf entries and an array without a
 * finite entry are REWL_ERR_ARG.  Temperatures are in units of J / k_B and must
 * be finite and > 0.  All arrays are caller-owned host memory. */

/* Canonical averages per spin (Sec. 3.1: the canonical distribution
 * P(E) ~ g(E) exp(-E/T) of Fig. 3b and its moments) at the nT temperatures
 * T[0 .. nT-1]: out[4i + 0] = u = <E> / N, out[4i + 1] = c = (<E^2> - <E>^2) /
 * (N T^2), out[4i + 2] = f = -T ln Z / N, out[4i + 3] = s = (u - f) / T, with
 * Z = sum_E g(E) exp(-E/T).  out holds 4 nT doubles. */
rewl_status rewl_canonical(const double *lng, size_t len, const double *T, size_t nT, double *out);

/* The canonical distribution at T scaled to 1 at its highest point (Fig. 3b
 * shows it normalised to 1 at the peaks): out[b] = P(E) / max P, 0 where
 * lng[b] = -INFINITY.  out holds len doubles. */
rewl_status rewl_canonical_distribution(const double *lng, size_t len, double T, double *out);

/* The largest specific heat c(T) (as rewl_canonical) for T in [T_lo, T_hi]:
 * a scan of 1025 temperatures, then a golden-section search between the best
 * one's neighbours down to 1e-13 T_hi.  *T_peak, *c_peak receive the maximum.
 * Errors: REWL_ERR_ARG (T_lo <= 0, T_hi <= T_lo, NULL output). */
rewl_status rewl_specific_heat_peak(const double *lng, size_t len, double T_lo, double T_hi, double *T_peak,
                                    double *c_peak);

/* The finite-size transition temperature Tc(L) of a first-order transition
 * (Sec. 3.1: 0.70126 for q = 10, L = 300; Fig. 3b): the temperature at which
 * the canonical distribution has two maxima of equal height.  Such pairs are
 * the successive vertices of the upper concave hull of (E, ln g(E)), at
 * T = 1 / slope of the edge between them; of the edges with T in
 * [T_lo, T_hi] the one spanning the widest energy range is taken (ties: the
 * lower one).  *Tc receives T; *e_low, *e_high (may be NULL) the energies of
 * the two peaks; *ln_suppression (may be NULL) ln of the smallest P(E) / P(peak)
 * between them (about ln 1e-14 for L = 300, Sec. 3.1).  Errors: REWL_ERR_STATE
 * when no edge has its temperature in the range. */
rewl_status rewl_equal_peak_temperature(const double *lng, size_t len, double T_lo, double T_hi, double *Tc,
                                        int *e_low, int *e_high, double *ln_suppression);

/* Join window pieces supplied by the caller into one normalised ln g: the
 * step rewl_get_lng applies to a run's own windows (Sec. 2, Fig. 2: each
 * neighbouring pair meets at the bin of their overlap where the pieces' slopes
 * d ln g / dE differ least; sum g = q^N).  e_lo[h]: lowest energy of each
 * window (increasing, inside [-2N, 0] with W); lng_w, mask_w: h x (W + 1),
 * window-major, mask 1 where the bin was visited; out: len = 2N + 1 doubles,
 * N = L * L.  Errors: REWL_ERR_ARG, REWL_ERR_STATE (a pair without a usable
 * joining bin). */
rewl_status rewl_join(int q, int L, int h, int W, const int *e_lo, const double *lng_w, const unsigned char *mask_w,
                      double *out, size_t len);

/* Bootstrap resampling of repeated runs (end of Sec. 2: the simulation is
 * repeated and resampled, and every resampled density of states is joined
 * anew, so its joining points move).  lng_runs, mask_runs: runs x h x (W + 1)
 * window pieces of `runs` runs of one geometry (e.g. rewl_get_field's
 * REWL_FIELD_LNG rows of walker 0 of every window, and REWL_FIELD_MASK).
 * Resample k takes the runs draws[k * runs .. k * runs + runs - 1] (indices in
 * [0, runs), drawn by the caller, repeats allowed), averages their pieces bin
 * by bin over the drawn runs that visited the bin (mask: visited by any), and
 * joins and normalises the averages as rewl_join into out[k * len .. ].  out
 * holds resamples x len doubles.  Errors as rewl_join, and REWL_ERR_ARG for a
 * draw outside [0, runs). */
rewl_status rewl_bootstrap(int q, int L, int h, int W, const int *e_lo, int runs, const double *lng_runs,
                           const unsigned char *mask_runs, int resamples, const int *draws, double *out, size_t len);

/* Device memory source for the handles, batches and servers created from now
 * on (no counterpart in the paper: it lets a framework's caching allocator, or
 * a fixed budget, supply the state arrays).  alloc(bytes, ctx) returns device
 * memory of the current device aligned to 256 bytes, or NULL; free(ptr, ctx)
 * takes back what alloc returned (NULL: the allocator keeps it).  alloc = NULL
 * restores cudaMalloc / cudaFree.  Each object frees its memory through the
 * allocator that gave it, so the source can change while objects live.  Not
 * safe to call while another thread creates objects.  A NULL return (or a
 * misaligned pointer) makes the creating call fail with REWL_ERR_NOMEM. */
void rewl_set_allocator(void *(*alloc)(size_t bytes, void *ctx), void (*free)(void *ptr, void *ctx), void *ctx);

/* Ising energy of the bin b = E + 2N of a q = 2 run (b broken bonds), in the
 * Ising convention E_I = -sum over bonds of s_i s_j (J = 1): each broken bond
 * counts +1 and each satisfied bond -1, so E_I = 2b - 2N = 2E + 2N with the
 * Potts energy E of Eq. 2 (for L = 8: E_I in [-128, 128], in steps of 4 where
 * g > 0).  *e_ising receives it.  Errors: REWL_ERR_ARG (L outside [3, 1024],
 * b outside [0, 2N], NULL output). */
rewl_status rewl_ising_energy(int L, int b, long long *e_ising);

/* Message of the last error on this thread ("" if none).  No counterpart in
 * the paper. */
const char *rewl_last_error(void);

/* Library version string.  No counterpart in the paper. */
const char *rewl_version(void);

/* ---- Measurement (no counterpart in the paper) ------------------------------
 * Issue rates of the pipes a WL step uses, measured on the current device by
 * micro-kernels (one CTA of 1024 threads per SM, eight independent chains of
 * one PTX operation per thread, timed with the SM clock): lane-operations per
 * clock per SM for add.rn.f64 (dadd), mad.lo.u32 (imad), mul.hi.u32
 * (imad_hi), lop3.b32 (lop3), add.u32 (iadd) and conflict-free ld.shared.u32
 * (lds); and the clocks of one dependent add.rn.f64, mad.lo.u32 and
 * ld.shared.u32.  The per-flip roofline of the benchmark divides these rates
 * by the method's per-flip operation counts.  Allocates and frees a few bytes
 * of device memory; synchronises the device.  Errors: REWL_ERR_ARG (NULL),
 * REWL_ERR_CUDA. */
typedef struct rewl_pipe_rates {
    double dadd, imad, imad_hi, lop3, iadd, lds;       /* per clock per SM  */
    double dadd_latency, imad_latency, lds_latency;    /* clocks            */
    int sms;                                           /* SMs of the device */
    double max_clock_mhz;                              /* its maximum clock */
} rewl_pipe_rates;
rewl_status rewl_measure_pipes(rewl_pipe_rates *out);

#ifdef __cplusplus
}
#endif

#endif /* REWL_H */
