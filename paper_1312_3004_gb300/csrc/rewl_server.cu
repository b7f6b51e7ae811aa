// rewl_server.cu -- continuous batching of density-of-states jobs.
//
// Jobs (REWL instances, Sec. 2 of arXiv:1312.3004) are submitted at any time.
// A job waits in a host queue until its device state fits into the server's
// memory pool (admission by footprint); admitted jobs stay resident on the
// device -- configurations, ln g, histograms; the random numbers are
// counter-based, so there is no generator state -- and every tick advances all
// resident jobs together with the batched kernels (one persistent sweep launch
// per spin-packing class, one batched check, one batched exchange per round).
// Converged jobs are retired at the end of a tick: their windows are joined on
// the host (Fig. 2), the result is kept, and their memory returns to the pool
// for the next admissions.  A job computes exactly the states it computes when
// run alone.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "rewl.h"
#include "rewl_host_internal.hpp"
#include "rewl_internal.cuh"

using rewl::host::fail;

namespace {

#define SRV_CUDA(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(REWL_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr int kWalkerThreads = 128;  // threads per CTA of the thread-per-walker sweep
constexpr long long kTuneMinWalkers = 512;  // below this, lane groups (a walker's chain sets the rate)

// First-fit allocator over one device arena (offsets in bytes, 256-aligned).
struct Arena {
    size_t size = 0;
    std::map<size_t, size_t> free_blocks;  // offset -> bytes
    void reset(size_t n) {
        size = n;
        free_blocks.clear();
        free_blocks[0] = n;
    }
    bool alloc(size_t n, size_t *off) {
        n = align256(n);
        for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n, at = it->first + n;
            free_blocks.erase(it);
            if (rest) free_blocks[at] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = align256(n);
        auto it = free_blocks.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_blocks.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_blocks.erase(nx);
        }
        if (it != free_blocks.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_blocks.erase(it);
            }
        }
    }
};

enum JobState { JOB_QUEUED = 0, JOB_RUNNING = 1, JOB_DONE = 2, JOB_FAILED = 3, JOB_CANCELLED = 4 };

struct Job {
    long long id = 0;
    rewl_params prm{};
    int spin_bits = 0;
    int state = JOB_QUEUED;
    rewl_s *inst = nullptr;  // while running
    size_t off = 0, bytes = 0;
    int slot = -1;  // control block slot while running
    double t_submit = 0, t_admit = 0, t_done = 0;
    long long rounds = 0, flips = 0;
    std::vector<double> result;  // joined, normalised ln g (2N + 1)
    rewl_status error = REWL_OK;
};

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct rewl_server_s {
    void *arena_mem = nullptr;
    rewl::host::DevBlock arena_block, ctl_block, tab_block;  // the device allocations
    Arena arena;
    int max_jobs = 0;
    rewl::Ctl *d_ctls = nullptr;  // [max_jobs] control blocks (one per slot)
    rewl::Ctl *h_ctls = nullptr;  // pinned mirrors
    std::vector<int> free_slots;
    cudaStream_t stream = nullptr;
    long long next_id = 1;
    std::map<long long, Job> jobs;
    std::vector<long long> queue;    // FIFO of queued job ids
    std::vector<long long> running;  // admitted, in table order
    bool tables_dirty = true;
    // device tables (grown on demand)
    void *d_tab = nullptr;
    size_t tab_cap = 0;
    rewl::InstDev *d_inst = nullptr;
    rewl::WinItem *d_wins = nullptr;
    int n_wins = 0;
    struct Cls {
        int bits = 4;
        std::vector<rewl::SweepItem> items;      // lane groups: walker groups of one job
        rewl::SweepItem *d_items = nullptr;
        int threads = 0, grid = 0;
        size_t smem = 0;
        std::vector<rewl::WalkerItem> walkers;   // a thread per walker: single walkers of any job
        rewl::WalkerItem *d_walkers = nullptr;
        int wgrid = 0;
    } cls[2];
    // How the resident walkers map to threads: 32 (lane groups, state staged in
    // shared memory) or 1 (a thread per walker, state in global memory).  Both
    // compute the same states; when the resident walker count has changed by
    // half since the last choice, the next two rounds time one mapping each and
    // the faster is kept.
    int lanes = 32;
    long long tuned_walkers = 0;
    unsigned int *d_queues = nullptr;
    int sms = 0, optin = 0;
    // counters
    long long rounds_run = 0, flips_done = 0;
};

namespace {

void finish_job(rewl_server_s *s, Job &j, int state) {
    if (j.inst) {
        s->arena.release(j.off, j.bytes);
        delete j.inst;
        j.inst = nullptr;
    }
    if (j.slot >= 0) s->free_slots.push_back(j.slot);
    j.slot = -1;
    j.state = state;
    j.t_done = now_s();
}

// Rebuild the device tables of the running jobs.
rewl_status rebuild_tables(rewl_server_s *s) {
    std::vector<rewl::InstDev> tab;
    std::vector<rewl::WinItem> wins;
    for (auto &c : s->cls) {
        c.items.clear();
        c.walkers.clear();
        c.threads = 32;
        c.smem = 0;
    }
    for (size_t i = 0; i < s->running.size(); ++i) {
        Job &j = s->jobs[s->running[i]];
        rewl_s *h = j.inst;
        rewl::InstDev d;
        d.M = h->M;
        d.S = h->S;
        d.lay = rewl::fast_layout(h->M, 32);
        tab.push_back(d);
        for (int w = 0; w < h->M.h; ++w) wins.push_back({(int)i, w});
        auto &c = s->cls[h->M.bits == 8 ? 1 : 0];
        int P = (int)((size_t)s->optin / (size_t)d.lay.stride);
        P = std::max(1, std::min(P, 8));
        for (int g0 = 0; g0 < h->M.G; g0 += P) c.items.push_back({(int)i, g0, std::min(P, h->M.G - g0), 0});
        for (int g = 0; g < h->M.G; ++g) c.walkers.push_back({(int)i, g});
        c.smem = std::max(c.smem, (size_t)P * (size_t)d.lay.stride);
        c.threads = std::max(c.threads, P * 32);
    }
    s->n_wins = (int)wins.size();
    const size_t need = align256(tab.size() * sizeof(rewl::InstDev) + 16) + align256(wins.size() * sizeof(rewl::WinItem) + 16) +
                        align256(s->cls[0].items.size() * sizeof(rewl::SweepItem) + 16) +
                        align256(s->cls[1].items.size() * sizeof(rewl::SweepItem) + 16) +
                        align256(s->cls[0].walkers.size() * sizeof(rewl::WalkerItem) + 16) +
                        align256(s->cls[1].walkers.size() * sizeof(rewl::WalkerItem) + 16) + 256;
    if (need > s->tab_cap) {
        SRV_CUDA(cudaStreamSynchronize(s->stream));
        rewl::host::dev_free(s->tab_block);
        s->d_tab = nullptr;
        s->tab_cap = std::max(need * 2, (size_t)(64 << 10));
        SRV_CUDA(rewl::host::dev_alloc(s->tab_block, s->tab_cap));
        s->d_tab = s->tab_block.ptr;
    }
    char *p = (char *)s->d_tab;
    s->d_inst = (rewl::InstDev *)p;
    p += align256(tab.size() * sizeof(rewl::InstDev) + 16);
    s->d_wins = (rewl::WinItem *)p;
    p += align256(wins.size() * sizeof(rewl::WinItem) + 16);
    for (auto &c : s->cls) {
        c.d_items = (rewl::SweepItem *)p;
        p += align256(c.items.size() * sizeof(rewl::SweepItem) + 16);
        c.d_walkers = (rewl::WalkerItem *)p;
        p += align256(c.walkers.size() * sizeof(rewl::WalkerItem) + 16);
    }
    s->d_queues = (unsigned int *)p;
    // the previous tables may still be read by queued rounds: order the copies
    // behind them on the same stream (copies from pageable memory are staged)
    SRV_CUDA(cudaStreamSynchronize(s->stream));
    if (!tab.empty())
        SRV_CUDA(cudaMemcpyAsync(s->d_inst, tab.data(), tab.size() * sizeof(rewl::InstDev), cudaMemcpyHostToDevice, s->stream));
    if (!wins.empty())
        SRV_CUDA(cudaMemcpyAsync(s->d_wins, wins.data(), wins.size() * sizeof(rewl::WinItem), cudaMemcpyHostToDevice, s->stream));
    for (int k = 0; k < 2; ++k) {
        auto &c = s->cls[k];
        c.bits = k == 1 ? 8 : 4;
        if (c.items.empty()) continue;
        SRV_CUDA(cudaMemcpyAsync(c.d_items, c.items.data(), c.items.size() * sizeof(rewl::SweepItem),
                                 cudaMemcpyHostToDevice, s->stream));
        SRV_CUDA(cudaMemcpyAsync(c.d_walkers, c.walkers.data(), c.walkers.size() * sizeof(rewl::WalkerItem),
                                 cudaMemcpyHostToDevice, s->stream));
        c.wgrid = (int)((c.walkers.size() + kWalkerThreads - 1) / kWalkerThreads);
        SRV_CUDA(rewl::launch_batch_sweep(c.bits, 32, nullptr, nullptr, 0, nullptr, 0, c.threads, c.smem, nullptr, true));
        const int per_sm = std::max(1, rewl::batch_sweep_ctas_per_sm(c.bits, 32, c.threads, c.smem));
        c.grid = std::min((int)c.items.size(), per_sm * s->sms);
    }
    SRV_CUDA(cudaStreamSynchronize(s->stream));
    s->tables_dirty = false;
    return REWL_OK;
}

rewl_status enqueue_round(rewl_server_s *s) {
    SRV_CUDA(cudaMemsetAsync(s->d_queues, 0, 2 * sizeof(unsigned int), s->stream));
    for (int k = 0; k < 2; ++k) {
        auto &c = s->cls[k];
        if (c.items.empty()) continue;
        if (s->lanes == 1)
            SRV_CUDA(rewl::launch_batch_walkers(c.bits, s->d_inst, c.d_walkers, (int)c.walkers.size(), c.wgrid,
                                                kWalkerThreads, s->stream, false));
        else
            SRV_CUDA(rewl::launch_batch_sweep(c.bits, 32, s->d_inst, c.d_items, (int)c.items.size(), s->d_queues + k,
                                              c.grid, c.threads, c.smem, s->stream, false));
    }
    SRV_CUDA(rewl::launch_batch_check(s->d_inst, s->d_wins, s->n_wins, s->stream));
    SRV_CUDA(rewl::launch_batch_exchange(s->d_inst, (int)s->running.size(), s->stream));
    return REWL_OK;
}

// Admit queued jobs (first fit in arrival order) while memory and slots allow.
rewl_status admit(rewl_server_s *s) {
    std::vector<long long> still;
    for (long long id : s->queue) {
        Job &j = s->jobs[id];
        if (j.state != JOB_QUEUED) continue;
        rewl_s *h = new rewl_s();
        h->owns = false;
        rewl_status st = rewl::host::prepare_instance(h, j.prm, j.spin_bits, 32);
        if (st) {
            delete h;
            j.error = st;
            finish_job(s, j, JOB_FAILED);
            continue;
        }
        size_t off = 0;
        if (s->free_slots.empty() || !s->arena.alloc(h->dbytes, &off)) {
            delete h;
            still.push_back(id);
            continue;
        }
        j.slot = s->free_slots.back();
        s->free_slots.pop_back();
        j.off = off;
        j.bytes = h->dbytes;
        rewl::host::carve_instance(h, (char *)s->arena_mem + off);
        h->S.ctl = s->d_ctls + j.slot;
        h->h_ctl = s->h_ctls + j.slot;
        h->stream = s->stream;
        SRV_CUDA(cudaMemsetAsync(h->S.ctl, 0, sizeof(rewl::Ctl), s->stream));
        SRV_CUDA(rewl::host::init_instance_async(h, s->stream));
        j.inst = h;
        j.state = JOB_RUNNING;
        j.t_admit = now_s();
        s->running.push_back(id);
        s->tables_dirty = true;
    }
    s->queue.swap(still);
    return REWL_OK;
}

}  // namespace

extern "C" {

rewl_status rewl_server_create(size_t pool_bytes, int max_jobs, rewl_server_t *out) {
    REWL_API_TRY
    if (!out || pool_bytes < 4096 || max_jobs < 1) return fail(REWL_ERR_ARG, "pool_bytes < 4096 or max_jobs < 1");
    *out = nullptr;
    rewl_server_s *s = new rewl_server_s();
    auto cleanup = [&](rewl_status st) {
        rewl_server_destroy(s);
        return st;
    };
    s->max_jobs = max_jobs;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&s->optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    pool_bytes = align256(pool_bytes);
    cudaError_t e = rewl::host::dev_alloc(s->arena_block, pool_bytes);
    if (e != cudaSuccess)
        return cleanup(fail(REWL_ERR_NOMEM, "device pool (%zu bytes): %s", pool_bytes, cudaGetErrorString(e)));
    s->arena_mem = s->arena_block.ptr;
    s->arena.reset(pool_bytes);
    e = rewl::host::dev_alloc(s->ctl_block, sizeof(rewl::Ctl) * (size_t)max_jobs);
    s->d_ctls = (rewl::Ctl *)s->ctl_block.ptr;
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_ctls, sizeof(rewl::Ctl) * (size_t)max_jobs);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(fail(REWL_ERR_NOMEM, "server set-up: %s", cudaGetErrorString(e)));
    for (int i = max_jobs - 1; i >= 0; --i) s->free_slots.push_back(i);
    *out = s;
    return REWL_OK;
    REWL_API_CATCH
}

void rewl_server_destroy(rewl_server_t s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (auto &kv : s->jobs)
        if (kv.second.inst) delete kv.second.inst;
    rewl::host::dev_free(s->tab_block);
    rewl::host::dev_free(s->ctl_block);
    if (s->h_ctls) cudaFreeHost(s->h_ctls);
    rewl::host::dev_free(s->arena_block);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

rewl_status rewl_server_submit(rewl_server_t s, const rewl_params *p, int spin_bits, long long *job_id) {
    REWL_API_TRY
    if (!s || !p) return fail(REWL_ERR_ARG, "NULL argument");
    rewl_s probe;
    rewl_status st = rewl::host::prepare_instance(&probe, *p, spin_bits, 32);
    if (st) return st;
    if (align256(probe.dbytes) > s->arena.size)
        return fail(REWL_ERR_NOMEM, "job needs %zu bytes; the pool holds %zu", probe.dbytes, s->arena.size);
    Job j;
    j.id = s->next_id++;
    j.prm = *p;
    j.spin_bits = spin_bits;
    j.t_submit = now_s();
    s->jobs[j.id] = j;
    s->queue.push_back(j.id);
    if (job_id) *job_id = j.id;
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_server_step(rewl_server_t s, long long rounds, int *n_running, int *n_queued) {
    REWL_API_TRY
    const rewl::host::Range range("rewl_server_step");
    if (!s) return fail(REWL_ERR_ARG, "NULL server");
    if (rounds < 1) return fail(REWL_ERR_ARG, "rounds < 1");
    rewl_status st = admit(s);
    if (st) return st;
    if (!s->running.empty()) {
        long long left = rounds;
        if (s->tables_dirty) {
            st = rebuild_tables(s);
            if (st) return st;
            long long walkers = 0;
            for (long long id : s->running) walkers += s->jobs[id].inst->M.G;
            if (walkers < kTuneMinWalkers) {
                s->lanes = 32;
                s->tuned_walkers = 0;
            } else if (s->tuned_walkers == 0 || 2 * walkers > 3 * s->tuned_walkers ||
                       3 * walkers < 2 * s->tuned_walkers) {
                // one round in each mapping, timed on the stream; the faster stays
                cudaEvent_t ev[3];
                for (auto &e : ev) SRV_CUDA(cudaEventCreate(&e));
                SRV_CUDA(cudaEventRecord(ev[0], s->stream));
                s->lanes = 32;
                st = enqueue_round(s);
                if (st == REWL_OK) SRV_CUDA(cudaEventRecord(ev[1], s->stream));
                s->lanes = 1;
                if (st == REWL_OK) st = enqueue_round(s);
                if (st == REWL_OK) SRV_CUDA(cudaEventRecord(ev[2], s->stream));
                float t32 = 0.0f, t1 = 0.0f;
                if (st == REWL_OK) SRV_CUDA(cudaEventSynchronize(ev[2]));
                if (st == REWL_OK) SRV_CUDA(cudaEventElapsedTime(&t32, ev[0], ev[1]));
                if (st == REWL_OK) SRV_CUDA(cudaEventElapsedTime(&t1, ev[1], ev[2]));
                for (auto &e : ev) cudaEventDestroy(e);
                if (st) return st;
                s->lanes = t1 < t32 ? 1 : 32;
                s->tuned_walkers = walkers;
                left -= 2;
            }
        }
        for (long long r = 0; r < left && st == REWL_OK; ++r) st = enqueue_round(s);
        if (st) return st;
        // status of every running job, then retire the converged ones
        for (long long id : s->running) {
            Job &j = s->jobs[id];
            SRV_CUDA(cudaMemcpyAsync(s->h_ctls + j.slot, s->d_ctls + j.slot, sizeof(rewl::Ctl), cudaMemcpyDeviceToHost,
                                     s->stream));
        }
        SRV_CUDA(cudaStreamSynchronize(s->stream));
        s->rounds_run += (left < rounds ? 2 : 0) + std::max(0LL, left);
        std::vector<long long> keep;
        for (long long id : s->running) {
            Job &j = s->jobs[id];
            const rewl::Ctl &c = s->h_ctls[j.slot];
            j.rounds = (long long)c.round;
            s->flips_done += (long long)c.flips - j.flips;
            j.flips = (long long)c.flips;
            if (c.error) {
                j.error = (c.error & rewl::ERR_OVERFLOW) ? REWL_ERR_OVERFLOW : REWL_ERR_STATE;
                finish_job(s, j, JOB_FAILED);
                s->tables_dirty = true;
            } else if (c.all_done) {
                j.result.assign((size_t)(2 * j.inst->M.N + 1), 0.0);
                st = rewl_get_lng(j.inst, j.result.data(), j.result.size(), 0);
                if (st) {
                    j.error = st;
                    j.result.clear();
                    finish_job(s, j, JOB_FAILED);
                } else {
                    finish_job(s, j, JOB_DONE);
                }
                s->tables_dirty = true;
            } else {
                keep.push_back(id);
            }
        }
        s->running.swap(keep);
    }
    if (n_running) *n_running = (int)s->running.size();
    if (n_queued) *n_queued = (int)s->queue.size();
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_server_mapping(rewl_server_t s, int *lanes, long long *tuned_walkers) {
    REWL_API_TRY
    if (!s) return fail(REWL_ERR_ARG, "NULL server");
    if (lanes) *lanes = s->lanes;
    if (tuned_walkers) *tuned_walkers = s->tuned_walkers;
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_server_poll(rewl_server_t s, long long job_id, int *state) {
    REWL_API_TRY
    if (!s || !state) return fail(REWL_ERR_ARG, "NULL argument");
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(REWL_ERR_ARG, "unknown job %lld", job_id);
    *state = it->second.state;
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_server_result(rewl_server_t s, long long job_id, double *out, size_t len) {
    REWL_API_TRY
    if (!s || !out) return fail(REWL_ERR_ARG, "NULL argument");
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(REWL_ERR_ARG, "unknown job %lld", job_id);
    const Job &j = it->second;
    if (j.state == JOB_FAILED) return fail(j.error ? j.error : REWL_ERR_STATE, "job %lld failed", job_id);
    if (j.state == JOB_CANCELLED) return fail(REWL_ERR_CANCELLED, "job %lld was cancelled", job_id);
    if (j.state != JOB_DONE) return fail(REWL_ERR_STATE, "job %lld has not finished", job_id);
    if (len != j.result.size()) return fail(REWL_ERR_ARG, "len %zu != 2N + 1 = %zu", len, j.result.size());
    std::memcpy(out, j.result.data(), len * sizeof(double));
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_server_job_info(rewl_server_t s, long long job_id, double *times, long long *counts) {
    REWL_API_TRY
    if (!s) return fail(REWL_ERR_ARG, "NULL server");
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(REWL_ERR_ARG, "unknown job %lld", job_id);
    const Job &j = it->second;
    if (times) {
        times[0] = j.t_submit;
        times[1] = j.t_admit;
        times[2] = j.t_done;
    }
    if (counts) {
        counts[0] = j.rounds;
        counts[1] = j.flips;
        counts[2] = (long long)j.bytes;
    }
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_server_cancel(rewl_server_t s, long long job_id) {
    REWL_API_TRY
    if (!s) return fail(REWL_ERR_ARG, "NULL server");
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(REWL_ERR_ARG, "unknown job %lld", job_id);
    Job &j = it->second;
    if (j.state == JOB_QUEUED) {
        s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), job_id), s->queue.end());
        finish_job(s, j, JOB_CANCELLED);
    } else if (j.state == JOB_RUNNING) {
        SRV_CUDA(cudaStreamSynchronize(s->stream));
        s->running.erase(std::remove(s->running.begin(), s->running.end(), job_id), s->running.end());
        finish_job(s, j, JOB_CANCELLED);
        s->tables_dirty = true;
    }
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_server_release(rewl_server_t s, long long job_id) {
    REWL_API_TRY
    if (!s) return fail(REWL_ERR_ARG, "NULL server");
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(REWL_ERR_ARG, "unknown job %lld", job_id);
    const int st = it->second.state;
    if (st == JOB_QUEUED || st == JOB_RUNNING)
        return fail(REWL_ERR_STATE, "job %lld is still %s", job_id, st == JOB_QUEUED ? "queued" : "running");
    s->jobs.erase(it);
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_server_info(rewl_server_t s, long long *counts, size_t *pool_free) {
    REWL_API_TRY
    if (!s) return fail(REWL_ERR_ARG, "NULL server");
    if (counts) {
        long long q = 0, r = 0, d = 0, f = 0;
        for (auto &kv : s->jobs) {
            const int st = kv.second.state;
            q += st == JOB_QUEUED;
            r += st == JOB_RUNNING;
            d += st == JOB_DONE;
            f += st == JOB_FAILED || st == JOB_CANCELLED;
        }
        counts[0] = q;
        counts[1] = r;
        counts[2] = d;
        counts[3] = f;
        counts[4] = s->rounds_run;
        counts[5] = s->flips_done;
    }
    if (pool_free) {
        size_t fr = 0;
        for (auto &kv : s->arena.free_blocks) fr += kv.second;
        *pool_free = fr;
    }
    return REWL_OK;
    REWL_API_CATCH
}

}  // extern "C"
