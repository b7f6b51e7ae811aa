// rewl_batch.cu -- many independent REWL instances of uneven size (q, L, h, m)
// in one device allocation, advanced together: one persistent sweep launch per
// (spin bits, lanes) class takes walker groups of every instance from a device
// queue, one batched check launch covers every window of every instance, one
// batched exchange launch every instance; a CUDA graph replays these rounds.
// Every instance computes exactly what it computes alone (its own Philox key,
// its own state; the kernels run the same block code as the single-instance
// launches).
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "rewl.h"
#include "rewl_host_internal.hpp"
#include "rewl_internal.cuh"

using rewl::host::fail;

namespace {

constexpr int kBatchGraphRounds = 4;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

#define BATCH_CUDA(call)                                                                        \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(REWL_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// A mapping of the batch's walkers to threads, and the spin packing: none of it
// changes a result (every choice runs the same block code on the same state).
struct Config {
    int bits = 8;           // spins per configuration word: 4 or 8 bits each
    int lanes = 32;         // 32: lane groups, state staged in shared memory; 1: a thread per walker
    int cta_kb = 72;        // lanes 32: shared memory per sweep CTA (walkers per CTA follow)
    int threads = 256;      // lanes 1: threads per CTA
};

struct SweepClass {
    int bits = 4, lanes = 32, threads = 0, grid = 0;
    size_t smem = 0;
    std::vector<rewl::SweepItem> items;      // lanes 32: groups of walkers of one instance
    rewl::SweepItem *d_items = nullptr;
    unsigned int *d_queue = nullptr;
    std::vector<rewl::WalkerItem> walkers;   // lanes 1: single walkers of any instance
    rewl::WalkerItem *d_walkers = nullptr;
};
// Batches of at least this many walkers in all run a thread per walker with its
// state in global memory (enough walkers to fill the SMs without lane groups),
// until rewl_batch_autotune measures otherwise.
constexpr long long kWalkerModeMin = 16384;

// Configurations the autotuner chose, by batch signature (process-wide).
std::mutex g_tune_mu;
std::map<std::string, Config> g_tune_cache;

}  // namespace

struct rewl_batch_s {
    std::vector<rewl_s *> inst;
    void *dmem = nullptr;         // instances and their control blocks
    rewl::host::DevBlock dblock;
    size_t dbytes = 0;
    rewl::Ctl *h_ctls = nullptr;  // pinned mirrors of every instance's control block
    rewl::Ctl *d_ctls = nullptr;  // the control blocks, contiguous
    cudaStream_t own_stream = nullptr, stream = nullptr;
    // tables of the current configuration (rebuilt by configure)
    rewl::host::DevBlock tblock;
    rewl::InstDev *d_inst = nullptr;
    rewl::WinItem *d_wins = nullptr;
    int n_wins = 0;
    std::vector<SweepClass> classes;
    unsigned int *d_queues = nullptr;
    cudaGraphExec_t graph = nullptr;
    int sms = 0;
    Config cfg;
    bool bits_free = false;   // the packing may change (spin_bits = 0 and every q <= 16)
    bool lanes_free = false;  // the mapping may change (lanes = 0)
    bool fits32[2] = {true, true};  // every walker fits a lane group's shared memory at 4 / 8 bits
    size_t bytes_config = 0;
};

namespace {

rewl_status enqueue_batch_round(rewl_batch_s *b, cudaStream_t s) {
    BATCH_CUDA(cudaMemsetAsync(b->d_queues, 0, sizeof(unsigned int) * b->classes.size(), s));
    for (auto &c : b->classes) {
        if (c.lanes == 1)
            BATCH_CUDA(rewl::launch_batch_walkers(c.bits, b->d_inst, c.d_walkers, (int)c.walkers.size(), c.grid,
                                                  c.threads, s, false));
        else
            BATCH_CUDA(rewl::launch_batch_sweep(c.bits, c.lanes, b->d_inst, c.d_items, (int)c.items.size(), c.d_queue,
                                                c.grid, c.threads, c.smem, s, false));
    }
    BATCH_CUDA(rewl::launch_batch_check(b->d_inst, b->d_wins, b->n_wins, s));
    BATCH_CUDA(rewl::launch_batch_exchange(b->d_inst, (int)b->inst.size(), s));
    return REWL_OK;
}

rewl_status build_batch_graph(rewl_batch_s *b) {
    cudaStream_t cap;
    BATCH_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    rewl_status st = REWL_OK;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int r = 0; r < kBatchGraphRounds && st == REWL_OK; ++r) st = enqueue_batch_round(b, cap);
        e = cudaStreamEndCapture(cap, &graph);
    }
    if (e == cudaSuccess && st == REWL_OK) e = cudaGraphInstantiate(&b->graph, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (st) return st;
    if (e != cudaSuccess) return fail(REWL_ERR_CUDA, "batch graph capture failed: %s", cudaGetErrorString(e));
    return REWL_OK;
}

rewl_status enqueue_batch_rounds(rewl_batch_s *b, long long n) {
    while (n >= kBatchGraphRounds) {
        BATCH_CUDA(cudaGraphLaunch(b->graph, b->stream));
        n -= kBatchGraphRounds;
    }
    for (; n > 0; --n) {
        rewl_status st = enqueue_batch_round(b, b->stream);
        if (st) return st;
    }
    return REWL_OK;
}

// Reads every control block; *done = number of converged instances.
rewl_status read_batch_status(rewl_batch_s *b, int *done) {
    const size_t n = b->inst.size();
    BATCH_CUDA(cudaMemcpyAsync(b->h_ctls, b->d_ctls, n * sizeof(rewl::Ctl), cudaMemcpyDeviceToHost, b->stream));
    BATCH_CUDA(cudaStreamSynchronize(b->stream));
    int d = 0;
    for (size_t i = 0; i < n; ++i) {
        const rewl::Ctl &c = b->h_ctls[i];
        if (c.error & rewl::ERR_OVERFLOW) return fail(REWL_ERR_OVERFLOW, "instance %zu: a histogram bin reached 2^31", i);
        if (c.error & rewl::ERR_ENTRY) return fail(REWL_ERR_STATE, "instance %zu: a walker could not enter its window", i);
        if (c.error & rewl::ERR_BOUNDS)
            return fail(REWL_ERR_STATE, "instance %zu: an index failed its bounds check (debug build)", i);
        d += c.all_done ? 1 : 0;
    }
    if (done) *done = d;
    return REWL_OK;
}

void destroy_batch(rewl_batch_s *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (rewl_s *h : b->inst) delete h;
    if (b->own_stream) cudaStreamDestroy(b->own_stream);
    if (b->h_ctls) cudaFreeHost(b->h_ctls);
    rewl::host::dev_free(b->tblock);
    rewl::host::dev_free(b->dblock);
    delete b;
}

// Spins of every instance repacked to `bits` per spin, in place: each
// instance's configurations are unpacked to bytes in a scratch buffer and
// packed again (the buffers were sized for 8-bit packing).
rewl_status repack(rewl_batch_s *b, int bits) {
    size_t need = 0;
    for (rewl_s *h : b->inst) need = std::max(need, (size_t)h->M.G * (size_t)h->M.N);
    rewl::host::DevBlock scratch;
    cudaError_t e = rewl::host::dev_alloc(scratch, need);
    if (e != cudaSuccess) return fail(REWL_ERR_NOMEM, "repacking scratch (%zu bytes): %s", need, cudaGetErrorString(e));
    for (rewl_s *h : b->inst) {
        if (h->M.bits == bits) continue;
        e = rewl::launch_get_spins(h->M, h->S, (uint8_t *)scratch.ptr, b->stream);
        if (e != cudaSuccess) break;
        h->M.bits = bits;
        h->M.wpc = (h->M.N * bits + 31) / 32;
        e = rewl::launch_set_spins(h->M, h->S, (const uint8_t *)scratch.ptr, b->stream);
        if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    rewl::host::dev_free(scratch);
    if (e != cudaSuccess) return fail(REWL_ERR_CUDA, "repacking: %s", cudaGetErrorString(e));
    return REWL_OK;
}

// Builds the tables, work lists, launch shapes and graph of configuration c
// (repacking the spins first if its packing differs).
rewl_status configure(rewl_batch_s *b, const Config &c) {
    BATCH_CUDA(cudaStreamSynchronize(b->stream));
    if (c.bits != b->cfg.bits || b->classes.empty()) {
        bool differ = false;
        for (rewl_s *h : b->inst) differ = differ || h->M.bits != c.bits;
        if (differ) {
            rewl_status st = repack(b, c.bits);
            if (st) return st;
        }
    }
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    const int n = (int)b->inst.size();
    std::vector<rewl::InstDev> tab((size_t)n);
    std::vector<rewl::WinItem> wins;
    for (int i = 0; i < n; ++i)
        for (int w = 0; w < b->inst[(size_t)i]->M.h; ++w) wins.push_back({i, w});
    b->n_wins = (int)wins.size();
    b->classes.clear();
    const size_t budget = (size_t)c.cta_kb * 1024;
    for (int i = 0; i < n; ++i) {
        rewl_s *h = b->inst[(size_t)i];
        tab[(size_t)i].M = h->M;
        tab[(size_t)i].S = h->S;
        tab[(size_t)i].lay = rewl::fast_layout(h->M, c.lanes, c.lanes == 1);
        int cls = -1;
        for (size_t k = 0; k < b->classes.size(); ++k)
            if (b->classes[k].bits == h->M.bits) cls = (int)k;
        if (cls < 0) {
            SweepClass sc;
            sc.bits = h->M.bits;
            sc.lanes = c.lanes;
            b->classes.push_back(sc);
            cls = (int)b->classes.size() - 1;
        }
        SweepClass &sc = b->classes[(size_t)cls];
        if (c.lanes == 1) {
            for (int g = 0; g < h->M.G; ++g) sc.walkers.push_back({i, g});
            continue;
        }
        const rewl::Layout &lay = tab[(size_t)i].lay;
        int P = (int)(std::max(budget, (size_t)lay.stride) / (size_t)lay.stride);
        P = std::min(P, 256 / sc.lanes);
        for (int g0 = 0; g0 < h->M.G; g0 += P) sc.items.push_back({i, g0, std::min(P, h->M.G - g0), 0});
        sc.smem = std::max(sc.smem, (size_t)P * (size_t)lay.stride);
        sc.threads = std::max(sc.threads, P * sc.lanes);
    }
    size_t off = 0;
    const size_t off_tab = off;
    off += align256((size_t)n * sizeof(rewl::InstDev));
    const size_t off_wins = off;
    off += align256(wins.size() * sizeof(rewl::WinItem));
    std::vector<size_t> off_items;
    for (auto &k : b->classes) {
        off_items.push_back(off);
        off += align256(k.lanes == 1 ? k.walkers.size() * sizeof(rewl::WalkerItem)
                                     : k.items.size() * sizeof(rewl::SweepItem));
    }
    const size_t off_q = off;
    off += align256(b->classes.size() * sizeof(unsigned int));
    rewl::host::dev_free(b->tblock);
    cudaError_t e = rewl::host::dev_alloc(b->tblock, off);
    if (e != cudaSuccess) return fail(REWL_ERR_NOMEM, "batch tables (%zu bytes): %s", off, cudaGetErrorString(e));
    b->bytes_config = off;
    char *base = (char *)b->tblock.ptr;
    b->d_inst = (rewl::InstDev *)(base + off_tab);
    b->d_wins = (rewl::WinItem *)(base + off_wins);
    b->d_queues = (unsigned int *)(base + off_q);
    e = cudaMemcpyAsync(b->d_inst, tab.data(), tab.size() * sizeof(rewl::InstDev), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_wins, wins.data(), wins.size() * sizeof(rewl::WinItem), cudaMemcpyHostToDevice, b->stream);
    for (size_t k = 0; k < b->classes.size() && e == cudaSuccess; ++k) {
        SweepClass &sc = b->classes[k];
        sc.d_queue = b->d_queues + k;
        if (sc.lanes == 1) {
            sc.d_walkers = (rewl::WalkerItem *)(base + off_items[k]);
            e = cudaMemcpyAsync(sc.d_walkers, sc.walkers.data(), sc.walkers.size() * sizeof(rewl::WalkerItem),
                                cudaMemcpyHostToDevice, b->stream);
            sc.threads = c.threads;
            sc.grid = (int)((sc.walkers.size() + (size_t)c.threads - 1) / (size_t)c.threads);
            continue;
        }
        sc.d_items = (rewl::SweepItem *)(base + off_items[k]);
        e = cudaMemcpyAsync(sc.d_items, sc.items.data(), sc.items.size() * sizeof(rewl::SweepItem),
                            cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) break;
        e = rewl::launch_batch_sweep(sc.bits, sc.lanes, nullptr, nullptr, 0, nullptr, 0, sc.threads, sc.smem, nullptr,
                                     true);
        if (e != cudaSuccess) break;
        const int per_sm = std::max(1, rewl::batch_sweep_ctas_per_sm(sc.bits, sc.lanes, sc.threads, sc.smem));
        sc.grid = std::min((int)sc.items.size(), per_sm * b->sms);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // tab and wins live on this frame
    if (e != cudaSuccess) return fail(REWL_ERR_CUDA, "batch configuration: %s", cudaGetErrorString(e));
    b->cfg = c;
    return build_batch_graph(b);
}

}  // namespace

extern "C" {

rewl_status rewl_batch_create(const rewl_params *jobs, int n, int spin_bits, rewl_batch_t *out) {
    REWL_API_TRY
    return rewl_batch_create_ext(jobs, n, spin_bits, 0, out);
    REWL_API_CATCH
}

rewl_status rewl_batch_create_ext(const rewl_params *jobs, int n, int spin_bits, int lanes, rewl_batch_t *out) {
    REWL_API_TRY
    if (!jobs || !out || n < 1) return fail(REWL_ERR_ARG, "NULL argument or n < 1");
    if (lanes != 0 && lanes != 1 && lanes != 32) return fail(REWL_ERR_ARG, "lanes %d not 0, 1 or 32", lanes);
    *out = nullptr;
    rewl_batch_s *b = new rewl_batch_s();
    auto cleanup = [&](rewl_status s) {
        destroy_batch(b);
        return s;
    };
    // ---- instances: parameters, sizes, plans -----------------------------------
    long long walkers = 0;
    bool small_q = true;
    for (int i = 0; i < n; ++i) {
        walkers += (long long)std::max(jobs[i].h, 0) * std::max(jobs[i].m, 0);
        small_q = small_q && jobs[i].q <= 16;
    }
    b->lanes_free = lanes == 0;
    b->bits_free = spin_bits == 0 && small_q;
    Config c;
    c.lanes = lanes != 0 ? lanes : (walkers >= kWalkerModeMin ? 1 : 32);
    // a thread per walker reads whole bytes faster than 4-bit fields
    c.bits = spin_bits != 0 ? spin_bits : ((c.lanes == 1 || !small_q) ? 8 : 4);
    size_t off = 0;
    std::vector<size_t> inst_off((size_t)n);
    for (int i = 0; i < n; ++i) {
        rewl_s *h = new rewl_s();
        h->owns = false;
        b->inst.push_back(h);
        rewl_status st = rewl::host::prepare_instance(h, jobs[i], c.bits, 32, b->bits_free ? 8 : 0);
        if (st) return cleanup(fail(st, "job %d: %s", i, rewl_last_error()));
        inst_off[(size_t)i] = off;
        off += align256(h->dbytes);
    }
    for (int i = 0; i < n; ++i) {  // a lane group's shared memory at either packing
        rewl_s *h = b->inst[(size_t)i];
        for (int k = 0; k < 2; ++k) {
            rewl::Model mk = h->M;
            mk.bits = k ? 8 : 4;
            mk.wpc = (mk.N * mk.bits + 31) / 32;
            if (rewl::fast_smem_per_walker(mk, 32) > (size_t)h->smem_optin) b->fits32[k] = false;
        }
    }
    if (c.lanes == 32 && !b->fits32[c.bits == 8]) {
        if (!b->lanes_free) return cleanup(fail(REWL_ERR_ARG, "a walker does not fit in shared memory"));
        c.lanes = 1;
    }
    b->sms = b->inst[0]->sms;
    const size_t off_ctl = off;
    off += align256((size_t)n * sizeof(rewl::Ctl));
    b->dbytes = off;
    cudaError_t e = rewl::host::dev_alloc(b->dblock, off);
    if (e != cudaSuccess)
        return cleanup(fail(REWL_ERR_NOMEM, "device memory (%zu bytes): %s", off, cudaGetErrorString(e)));
    b->dmem = b->dblock.ptr;
    e = cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(fail(REWL_ERR_CUDA, "stream: %s", cudaGetErrorString(e)));
    b->stream = b->own_stream;
    e = cudaMallocHost(&b->h_ctls, (size_t)n * sizeof(rewl::Ctl));
    if (e != cudaSuccess) return cleanup(fail(REWL_ERR_NOMEM, "cudaMallocHost: %s", cudaGetErrorString(e)));
    char *base = (char *)b->dmem;
    b->d_ctls = (rewl::Ctl *)(base + off_ctl);
    // ---- carve and initialise every instance ---------------------------------
    e = cudaMemsetAsync(b->d_ctls, 0, (size_t)n * sizeof(rewl::Ctl), b->stream);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        rewl_s *h = b->inst[(size_t)i];
        rewl::host::carve_instance(h, base + inst_off[(size_t)i]);
        h->S.ctl = b->d_ctls + i;  // control blocks contiguous: one status read for all
        h->stream = b->stream;
        h->h_ctl = b->h_ctls + i;
        e = rewl::host::init_instance_async(h, b->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cleanup(fail(REWL_ERR_CUDA, "batch set-up: %s", cudaGetErrorString(e)));
    rewl_status st = read_batch_status(b, nullptr);
    if (st) return cleanup(st);
    b->cfg = c;
    st = configure(b, c);
    if (st) return cleanup(st);
    *out = b;
    return REWL_OK;
    REWL_API_CATCH
}

void rewl_batch_destroy(rewl_batch_t b) { destroy_batch(b); }

rewl_status rewl_batch_autotune(rewl_batch_t b, int rounds, rewl_tune_entry *entries, int max_entries,
                                int *n_entries, int *from_cache) {
    REWL_API_TRY
    const rewl::host::Range range("rewl_batch_autotune");
    if (!b) return fail(REWL_ERR_ARG, "NULL batch");
    if (max_entries < 0 || (max_entries > 0 && !entries)) return fail(REWL_ERR_ARG, "entries");
    if (n_entries) *n_entries = 0;
    if (from_cache) *from_cache = 0;
    // the batch's signature: device, freedoms, and every instance's shape
    std::string key = std::to_string(b->sms) + (b->bits_free ? "b" : "B") + (b->lanes_free ? "l" : "L") +
                      std::to_string(b->cfg.bits) + "/" + std::to_string(b->cfg.lanes);
    for (rewl_s *h : b->inst)
        key += ";" + std::to_string(h->M.q) + "," + std::to_string(h->M.L) + "," + std::to_string(h->M.h) + "," +
               std::to_string(h->M.m) + "," + std::to_string(h->M.K);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end() && rounds <= 0) {
            if (from_cache) *from_cache = 1;
            return configure(b, it->second);
        }
    }
    if (rounds <= 0) rounds = 2;
    std::vector<Config> cands;
    const int bits_opts[2] = {b->cfg.bits, b->cfg.bits == 8 ? 4 : 8};
    for (int bi = 0; bi < (b->bits_free ? 2 : 1); ++bi) {
        const int bits = bits_opts[bi];
        const int lane_opts[2] = {b->cfg.lanes, b->cfg.lanes == 32 ? 1 : 32};
        for (int li = 0; li < (b->lanes_free ? 2 : 1); ++li) {
            const int lanes = lane_opts[li];
            if (lanes == 32 && !b->fits32[bits == 8]) continue;
            Config c;
            c.bits = bits;
            c.lanes = lanes;
            if (lanes == 32) {
                for (int kb : {36, 72, 110}) {
                    c.cta_kb = kb;
                    cands.push_back(c);
                }
            } else {
                for (int t : {128, 256}) {
                    c.threads = t;
                    cands.push_back(c);
                }
            }
        }
    }
    cudaEvent_t e0, e1;
    BATCH_CUDA(cudaEventCreate(&e0));
    BATCH_CUDA(cudaEventCreate(&e1));
    int best = -1, n_done = 0;
    double best_rate = -1.0;
    rewl_status st = REWL_OK;
    int n_conv = 0;
    for (size_t i = 0; i < cands.size() && st == REWL_OK; ++i) {
        st = configure(b, cands[i]);
        if (st) break;
        st = enqueue_batch_rounds(b, 1);  // settles the new configuration
        if (st == REWL_OK) st = read_batch_status(b, &n_conv);
        if (st) break;
        unsigned long long f0 = 0, f1 = 0;
        for (size_t k = 0; k < b->inst.size(); ++k) f0 += b->h_ctls[k].flips;
        cudaError_t e = cudaEventRecord(e0, b->stream);
        if (e == cudaSuccess) st = enqueue_batch_rounds(b, rounds);
        if (e == cudaSuccess && st == REWL_OK) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess && st == REWL_OK) st = read_batch_status(b, &n_conv);
        float ms = 0.0f;
        if (e == cudaSuccess && st == REWL_OK) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess && st == REWL_OK) st = fail(REWL_ERR_CUDA, "autotune timing: %s", cudaGetErrorString(e));
        if (st) break;
        for (size_t k = 0; k < b->inst.size(); ++k) f1 += b->h_ctls[k].flips;
        const double rate = ms > 0.0f ? (double)(f1 - f0) / (ms * 1e-3) : 0.0;
        if (n_done < max_entries) {
            rewl_tune_entry &en = entries[n_done];
            en.spin_bits = cands[i].bits;
            en.lanes = cands[i].lanes;
            en.cta_kb = cands[i].lanes == 32 ? cands[i].cta_kb : 0;
            en.threads = cands[i].lanes == 1 ? cands[i].threads : 0;
            en.flips_per_s = rate;
        }
        ++n_done;
        if (rate > best_rate) {
            best_rate = rate;
            best = (int)i;
        }
        if (n_conv == (int)b->inst.size()) break;  // nothing left to time
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    if (n_entries) *n_entries = std::min(n_done, max_entries);
    if (best < 0) return REWL_OK;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = cands[(size_t)best];
    }
    return configure(b, cands[(size_t)best]);
    REWL_API_CATCH
}

rewl_status rewl_batch_config(rewl_batch_t b, int *spin_bits, int *lanes, int *cta_kb, int *threads) {
    REWL_API_TRY
    if (!b) return fail(REWL_ERR_ARG, "NULL batch");
    if (spin_bits) *spin_bits = b->cfg.bits;
    if (lanes) *lanes = b->cfg.lanes;
    if (cta_kb) *cta_kb = b->cfg.lanes == 32 ? b->cfg.cta_kb : 0;
    if (threads) *threads = b->cfg.lanes == 1 ? b->cfg.threads : 0;
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_batch_set_stream(rewl_batch_t b, void *stream) {
    REWL_API_TRY
    if (!b) return fail(REWL_ERR_ARG, "NULL batch");
    BATCH_CUDA(cudaStreamSynchronize(b->stream));
    b->stream = stream ? (cudaStream_t)stream : b->own_stream;
    for (rewl_s *h : b->inst) h->stream = b->stream;
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_batch_run_async(rewl_batch_t b, long long rounds) {
    REWL_API_TRY
    if (!b) return fail(REWL_ERR_ARG, "NULL batch");
    if (rounds < 0) return fail(REWL_ERR_ARG, "rounds < 0");
    return enqueue_batch_rounds(b, rounds);
    REWL_API_CATCH
}

rewl_status rewl_batch_sync(rewl_batch_t b, int *n_converged) {
    REWL_API_TRY
    if (!b) return fail(REWL_ERR_ARG, "NULL batch");
    return read_batch_status(b, n_converged);
    REWL_API_CATCH
}

rewl_status rewl_batch_run(rewl_batch_t b, long long max_rounds, int *n_converged) {
    REWL_API_TRY
    const rewl::host::Range range("rewl_batch_run");
    if (!b) return fail(REWL_ERR_ARG, "NULL batch");
    const int n = (int)b->inst.size();
    int done = 0;
    rewl_status st = read_batch_status(b, &done);
    long long left = max_rounds;
    while (st == REWL_OK && done < n && (max_rounds <= 0 || left > 0)) {
        const long long k = (max_rounds <= 0 || left >= kBatchGraphRounds) ? kBatchGraphRounds : left;
        st = enqueue_batch_rounds(b, k);
        if (st == REWL_OK) st = read_batch_status(b, &done);
        left -= k;
    }
    if (n_converged) *n_converged = done;
    return st;
    REWL_API_CATCH
}

rewl_status rewl_batch_instance(rewl_batch_t b, int i, rewl_t *view) {
    REWL_API_TRY
    if (!b || !view) return fail(REWL_ERR_ARG, "NULL argument");
    if (i < 0 || i >= (int)b->inst.size()) return fail(REWL_ERR_ARG, "instance %d outside [0, %zu)", i, b->inst.size());
    *view = b->inst[(size_t)i];
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_batch_info(rewl_batch_t b, int *n_instances, long long *walkers, size_t *device_bytes) {
    REWL_API_TRY
    if (!b) return fail(REWL_ERR_ARG, "NULL batch");
    long long w = 0;
    for (rewl_s *h : b->inst) w += h->M.G;
    if (n_instances) *n_instances = (int)b->inst.size();
    if (walkers) *walkers = w;
    if (device_bytes) *device_bytes = b->dbytes;
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_batch_stats(rewl_batch_t b, rewl_stats *s) {
    REWL_API_TRY
    if (!b || !s) return fail(REWL_ERR_ARG, "NULL argument");
    int done = 0;
    rewl_status st = read_batch_status(b, &done);
    std::memset(s, 0, sizeof *s);
    s->min_lnf = 0.0;
    s->max_lnf = 0.0;
    for (size_t i = 0; i < b->inst.size(); ++i) {
        const rewl::Ctl &c = b->h_ctls[i];
        s->rounds = std::max(s->rounds, (long long)c.round);
        s->flips += (long long)c.flips;
        s->accepted += (long long)c.accepted;
        s->exch_tried += (long long)c.xtried;
        s->exch_accepted += (long long)c.xacc;
        s->near_ties += (long long)c.ties;
        s->slow_decisions += (long long)c.slow;
        s->seq_steps += (long long)c.seq;
    }
    s->windows_done = done;  // instances, for a batch
    s->converged = done == (int)b->inst.size() ? 1 : 0;
    return st;
    REWL_API_CATCH
}

}  // extern "C"
