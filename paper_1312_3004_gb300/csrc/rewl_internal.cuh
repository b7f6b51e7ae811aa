// rewl_internal.cuh -- device state layout and kernel launchers shared by the
// kernels (rewl_kernels.cu) and the host driver (rewl_host.cu).
//
// Device state of one REWL instance (Sec. 2 of arXiv:1312.3004): h windows of
// m walkers, G = h*m walker slots, C = G configuration buffers.  A walker slot
// g = i*m + k owns ln g and H of window i; the configuration it carries is the
// buffer slot_cfg[g], so a replica exchange swaps two 32-bit buffer ids instead
// of two lattices, and the buffer id doubles as the replica id.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rewl {

// Device control block: round counter, completion and error flags, counters.
struct Ctl {
    unsigned long long round;     // exchange rounds completed
    unsigned int all_done;        // every window has ln f < ln f_final
    unsigned int error;           // ERR_* bits
    unsigned long long flips;     // WL proposals
    unsigned long long accepted;  // accepted WL proposals
    unsigned long long xtried;    // exchange pairs evaluated
    unsigned long long xacc;      // exchanges carried out
    unsigned long long ties;      // |u - exp(D)| < 1e-14 acceptance draws
    unsigned long long slow;      // WL decisions resolved on the FP64 path
    unsigned long long seq;       // WL steps the fast sweep resolved one at a time
};

enum : unsigned int {
    ERR_OVERFLOW = 1u,  // an H bin reached 2^31
    ERR_ENTRY = 2u,     // a walker could not reach its window
    ERR_BOUNDS = 4u,    // debug build: an index failed its bounds check
    ERR_ENERGY = 8u,    // debug build: a kept energy differs from its recount
};

// Bounds checks of the debug build (REWL_DEBUG_CHECKS): an index outside
// [lo, hi) counts into `bad` and is replaced by lo, so the access stays inside
// the array and the kernel finishes; the caller raises ERR_BOUNDS.  In the
// release build the index passes through unchanged.
#ifdef REWL_DEBUG_CHECKS
__device__ __forceinline__ int checked_index(int i, int lo, int hi, unsigned int &bad) {
    if (i < lo || i >= hi) {
        ++bad;
        return lo;
    }
    return i;
}
#define REWL_IDX(i, lo, hi, bad) rewl::checked_index((i), (lo), (hi), (bad))
#else
#define REWL_IDX(i, lo, hi, bad) (i)
#endif

// Random-number domains: the fourth Philox counter word.
enum : uint32_t { DOM_WL = 0, DOM_INIT = 1, DOM_ENTRY = 2, DOM_PERM = 3, DOM_XACC = 4 };

struct Model {
    int q, L, N, W, B;        // B = W + 1 bins per window
    int h, m, G;              // windows, walkers per window, walker slots
    int bits;                 // 4 or 8 bits per stored spin
    int wpc;                  // 32-bit words per configuration buffer
    uint32_t key0, key1;      // Philox key = seed
    uint32_t divL;            // ceil(2^32 / L) for site -> (x, y)
    long long K;              // WL steps per walker between exchanges
    double lnf_final, flatness;
    int schedule;             // ln f schedule: SCHED_HALVING or SCHED_INV_T
    int production;           // 1: fixed-weight production (ln f = 0, H(E,O) kept, every window runs)
    int n_obins;              // production: classes of the majority count O
};

// ln f schedules of the window check: halving per iteration (Sec. 2), or the
// 1/t rule (Belardinelli & Pereyra), which Sec. 2 admits as another valid WL
// update rule.
enum : int { SCHED_HALVING = 0, SCHED_INV_T = 1 };

struct State {
    uint32_t *spins;      // [G][wpc] packed configurations, by buffer id
    int32_t *cfg_E;       // [G] energy of each configuration buffer
    uint32_t *slot_cfg;   // [G] buffer held by walker slot g (its replica id)
    unsigned long long *t;// [G] WL steps of walker slot g
    double *lng;          // [G][B] ln g of walker slot g
    uint32_t *H;          // [G][B] histogram of walker slot g
    uint8_t *mask;        // [h][B] bins visited by any walker of the window
    int32_t *e_lo;        // [h] lowest energy of each window
    double *lnf;          // [h] ln f of each window
    int32_t *iter;        // [h] completed iterations
    uint8_t *done;        // [h] window finished
    uint8_t *rt_end;      // [G] by replica id: last end of the energy range its window touched (0, 1 low, 2 high)
    uint32_t *rt_trips;   // [G] by replica id: completed round trips (lowest window -> highest -> lowest)
    long long *shadow;    // [G][B + 2 kShadowPad] ln g shadows of the one-lane sweep that keeps
                          // every walker's state in global memory
    uint8_t *phase;       // [h] 1/t rule: 1 once the window follows ln f = 1/t
    unsigned long long *tlog;  // [kTieLog][2] the first near-tie decisions: (kind << 32 | who, when)
    unsigned long long *heo;   // production: [h][B][n_obins] visits H(E, O) of each window
    int32_t *cnt;              // production: [G][q] spins of each value, by configuration buffer
    Ctl *ctl;             // control block
};

// Near-tie log.  An acceptance draw with |u - exp(D)| < 1e-14 is one where the
// exp of two libraries can decide differently; each is counted in Ctl::ties and
// the first kTieLog are recorded, so that a GPU / CPU difference can be traced
// to the decision that caused it.  Kinds: a WL step (who = walker slot g, when
// = its step index t) or an exchange (who = slot of the lower window's walker,
// when = the exchange round).
constexpr int kTieLog = 32;
enum : unsigned int { TIE_WL = 0u, TIE_EXCHANGE = 1u };
__device__ __forceinline__ void record_tie(Ctl *ctl, unsigned long long *tlog, unsigned int kind, unsigned int who,
                                           unsigned long long when) {
    const unsigned long long i = atomicAdd(&ctl->ties, 1ull);
    if (i < (unsigned long long)kTieLog) {
        tlog[2 * i] = ((unsigned long long)kind << 32) | who;
        tlog[2 * i + 1] = when;
    }
}

enum : int { SWEEP_REFERENCE = 0, SWEEP_FAST = 1 };

// Shared-memory layout of one walker in the fast sweep.  The binary64 ln g and
// the histogram stay in global memory (L2); off_lat < 0: so does the lattice.
struct Layout {
    int stride;                 // bytes per walker (multiple of 16)
    int off_lgf, off_lat;       // byte offsets: ln g shadow (with sentinels), lattice
    int off_q, off_e, off_bm;   // serial-loop staging and conflict marks (lane groups)
};

// One instance of a batch, as the batched kernels see it.
struct InstDev {
    Model M;
    State S;
    Layout lay;   // fast-sweep layout of this instance's walkers
};
// A piece of sweep work: P walkers g0 .. g0 + P - 1 of one instance.
struct SweepItem {
    int inst, g0, P, pad;
};
// One walker of one instance (the batched one-lane sweep: a thread per walker).
struct WalkerItem {
    int inst, g;
};
// A window of one instance for the batched check.
struct WinItem {
    int inst, w;
};

struct SweepPlan {
    int kind;        // SWEEP_REFERENCE (binary64 on the chain) or SWEEP_FAST
    int lanes;       // lanes per walker of the fast sweep (1, 2, 4, 8, 16, 32)
    int P;           // walkers per CTA
    int threads;     // CTA size
    int grid;        // CTAs
    size_t smem;     // dynamic shared memory bytes
    int lat_global;  // fast sweep: the lattice stays in global memory (large lattices)
};

// Launchers (rewl_kernels.cu).  All enqueue on `s` and return the launch error.
cudaError_t launch_init(const Model &M, const State &S, cudaStream_t s);
// kind: SWEEP_REFERENCE / SWEEP_FAST; lanes: 0 = choose from the walker count.
// A plan with P == 0 means the configuration does not fit (shared memory).
// lat_mode: where the fast sweep keeps the lattices (0 by size, 1 global, 2 shared).
SweepPlan plan_sweep(const Model &M, int num_sms, size_t smem_optin, int kind = SWEEP_FAST, int lanes = 0,
                     int lat_mode = 0);
cudaError_t prepare_sweep(const Model &M, const SweepPlan &p);
cudaError_t launch_sweep(const Model &M, const State &S, const SweepPlan &p, cudaStream_t s);
cudaError_t launch_window_check(const Model &M, const State &S, cudaStream_t s);
cudaError_t launch_exchange(const Model &M, const State &S, cudaStream_t s);
// Fixed-weight production (M.production = 1): the spin counts of every
// configuration buffer, and K Metropolis steps with weights 1/g(E) per walker
// with H(E, O) accumulated per window.
cudaError_t launch_count_spins(const Model &M, const State &S, cudaStream_t s);
cudaError_t launch_production_sweep(const Model &M, const State &S, cudaStream_t s);
cudaError_t launch_set_spins(const Model &M, const State &S, const uint8_t *spins_dev, cudaStream_t s);
cudaError_t launch_get_spins(const Model &M, const State &S, uint8_t *spins_dev, cudaStream_t s);
size_t sweep_smem_per_walker(const Model &M);
size_t fast_smem_per_walker(const Model &M, int lanes, bool lat_global = false);
cudaError_t launch_sweep_fast(const Model &M, const State &S, const SweepPlan &p, cudaStream_t s, bool prepare);

Layout fast_layout(const Model &M, int lanes, bool lat_global = false);
// A lattice above this many bytes stays in global memory in the fast sweep.
constexpr int kSharedLatticeMax = 16384;
// Sentinel bins beyond each end of a window in the ln g shadow.
constexpr int kShadowPad = 24;
// The batched one-lane sweep: every walker's state in global memory, a thread
// per walker, walkers of any instances of one spin packing in a CTA.
cudaError_t launch_batch_walkers(int bits, const InstDev *inst, const WalkerItem *items, int n_items, int grid,
                                 int threads, cudaStream_t s, bool prepare);
int batch_walkers_ctas_per_sm(int bits, int threads);
cudaError_t launch_batch_check(const InstDev *inst, const WinItem *wins, int n_wins, cudaStream_t s);
cudaError_t launch_batch_exchange(const InstDev *inst, int n_inst, cudaStream_t s);
// Persistent batched sweep for one (spin bits, lanes) class: CTAs of `threads`
// threads with `smem` bytes take items from *queue until n_items are done.
cudaError_t launch_batch_sweep(int bits, int lanes, const InstDev *inst, const SweepItem *items, int n_items,
                               unsigned int *queue, int grid, int threads, size_t smem, cudaStream_t s,
                               bool prepare);
int batch_sweep_ctas_per_sm(int bits, int lanes, int threads, size_t smem);

// Record the message returned by rewl_last_error() on this thread (rewl_host.cu).
void set_error(const char *msg);

}  // namespace rewl
