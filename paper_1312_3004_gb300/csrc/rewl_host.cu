// rewl_host.cu -- host driver behind include/rewl.h: parameter checks, the
// window table, device state, the round loop as a CUDA graph, state access,
// joining of the windows' pieces (Sec. 2, Fig. 2) and save / load.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rewl.h"
#include "rewl_host_internal.hpp"
#include "rewl_internal.cuh"

using rewl::Ctl;
using rewl::Model;
using rewl::State;

namespace {

thread_local std::string g_last_error;

rewl_status fail(rewl_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

#define REWL_CUDA(call)                                                                        \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(REWL_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));        \
    } while (0)

// Rounds per captured graph: one replay queues this many (sweep, check,
// exchange) triples; the host polls the completion flag between replays.
constexpr int kGraphRounds = 8;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Window table (Sec. 2, Fig. 1): h equal windows of W + 1 bins covering
// [-2N, 0] with overlap o.  W = ceil(2N / (1 + (h-1)(1-o))); window i starts
// at -2N + round_half_up(i (2N - W) / (h - 1)).
bool window_geometry(int L, int h, double o, std::vector<int32_t> &e_lo, int &W) {
    const long long N = (long long)L * L, R = 2 * N;
    const double span = 1.0 + (double)(h - 1) * (1.0 - o);
    long long w = (long long)std::ceil((double)R / span);
    if (w > R) w = R;
    if (w < 8) return false;
    e_lo.assign((size_t)h, 0);
    for (int i = 0; i < h; ++i) {
        const long long off = h > 1 ? (2LL * i * (R - w) + (h - 1)) / (2LL * (h - 1)) : 0LL;
        e_lo[(size_t)i] = (int32_t)(-2 * N + off);
    }
    W = (int)w;
    return true;
}

}  // namespace

void rewl::set_error(const char *msg) { g_last_error = msg; }

rewl_status rewl::host::fail(rewl_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}



namespace {

rewl_status check_params(const rewl_params &p, int spin_bits) {
    if (p.q < 2 || p.q > 255) return fail(REWL_ERR_ARG, "q=%d outside [2, 255]", p.q);
    if (p.L < 3 || p.L > 1024) return fail(REWL_ERR_ARG, "L=%d outside [3, 1024]", p.L);
    if (p.h < 1) return fail(REWL_ERR_ARG, "h=%d < 1", p.h);
    if (!(p.overlap >= 0.0 && p.overlap < 1.0)) return fail(REWL_ERR_ARG, "overlap %g outside [0, 1)", p.overlap);
    if (p.m < 1 || p.m > 256) return fail(REWL_ERR_ARG, "m=%d outside [1, 256]", p.m);
    if (!(p.lnf_final > 0.0 && p.lnf_final < 1.0)) return fail(REWL_ERR_ARG, "lnf_final %g outside (0, 1)", p.lnf_final);
    if (!(p.flatness > 0.0 && p.flatness < 1.0)) return fail(REWL_ERR_ARG, "flatness %g outside (0, 1)", p.flatness);
    if (p.exchange_interval < 1) return fail(REWL_ERR_ARG, "exchange_interval %lld < 1", p.exchange_interval);
    if (spin_bits != 0 && spin_bits != 4 && spin_bits != 8) return fail(REWL_ERR_ARG, "spin_bits %d not 0, 4 or 8", spin_bits);
    if (spin_bits == 4 && p.q > 16) return fail(REWL_ERR_ARG, "4-bit spins need q <= 16");
    if ((long long)p.h * p.m > (1LL << 30)) return fail(REWL_ERR_ARG, "too many walkers");
    return REWL_OK;
}

rewl_status enqueue_round(rewl_s *h, cudaStream_t s) {
    REWL_CUDA(rewl::launch_sweep(h->M, h->S, h->plan, s));
    REWL_CUDA(rewl::launch_window_check(h->M, h->S, s));
    REWL_CUDA(rewl::launch_exchange(h->M, h->S, s));
    return REWL_OK;
}

rewl_status build_graph(rewl_s *h) {
    cudaStream_t cap;
    REWL_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    rewl_status st = REWL_OK;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int r = 0; r < kGraphRounds && st == REWL_OK; ++r) st = enqueue_round(h, cap);
        e = cudaStreamEndCapture(cap, &graph);
    }
    if (e == cudaSuccess && st == REWL_OK) e = cudaGraphInstantiate(&h->graph, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (st != REWL_OK) return st;
    if (e != cudaSuccess) return fail(REWL_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    return REWL_OK;
}

rewl_status enqueue_rounds(rewl_s *h, long long n) {
    while (n >= kGraphRounds) {
        REWL_CUDA(cudaGraphLaunch(h->graph, h->stream));
        n -= kGraphRounds;
    }
    for (; n > 0; --n) {
        rewl_status st = enqueue_round(h, h->stream);
        if (st) return st;
    }
    return REWL_OK;
}

rewl_status read_ctl(rewl_s *h) {
    REWL_CUDA(cudaMemcpyAsync(h->h_ctl, h->S.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
    REWL_CUDA(cudaStreamSynchronize(h->stream));
    if (h->h_ctl->error & rewl::ERR_OVERFLOW) return fail(REWL_ERR_OVERFLOW, "a histogram bin reached 2^31 visits");
    if (h->h_ctl->error & rewl::ERR_ENTRY) return fail(REWL_ERR_STATE, "a walker could not enter its window");
    if (h->h_ctl->error & rewl::ERR_BOUNDS) return fail(REWL_ERR_STATE, "an index failed its bounds check (debug build)");
    if (h->h_ctl->error & rewl::ERR_ENERGY)
        return fail(REWL_ERR_STATE, "a walker's energy differs from its recount (debug build)");
    return REWL_OK;
}

}  // namespace

// ---- joining (Sec. 2, Fig. 2) ------------------------------------------------
namespace rewl {
namespace host {

// Slope of a piece at local bin i: difference quotient between the nearest
// visited bins below and above i (i itself must be visited).
bool piece_slope(const double *lg, const uint8_t *vis, int B, int i, double *beta) {
    if (!vis[i]) return false;
    int a = i - 1;
    while (a >= 0 && !vis[a]) --a;
    int b = i + 1;
    while (b < B && !vis[b]) ++b;
    if (a < 0 || b >= B) return false;
    *beta = (lg[b] - lg[a]) / (double)(b - a);
    return true;
}

rewl_status join_windows(int N, int W, const std::vector<int32_t> &e_lo, const std::vector<double> &lw,
                         const std::vector<uint8_t> &mw, double *out) {
    const int h = (int)e_lo.size(), B = W + 1, nb = 2 * N + 1;
    std::vector<double> offset((size_t)h, 0.0);
    std::vector<int> cut((size_t)h, 0);
    int last = -1;
    for (int a = 0; a + 1 < h; ++a) {
        const int lo_a = e_lo[(size_t)a] + 2 * N, lo_b = e_lo[(size_t)a + 1] + 2 * N;
        const double *pa = &lw[(size_t)a * B], *pb = &lw[(size_t)(a + 1) * B];
        const uint8_t *va = &mw[(size_t)a * B], *vb = &mw[(size_t)(a + 1) * B];
        int join = -1;
        double gap = 0.0;
        for (int b = std::max(lo_b, last + 1); b <= lo_a + W; ++b) {
            double ba, bb;
            if (!piece_slope(pa, va, B, b - lo_a, &ba) || !piece_slope(pb, vb, B, b - lo_b, &bb)) continue;
            const double d = std::fabs(ba - bb);
            if (join < 0 || d < gap) {
                join = b;
                gap = d;
            }
        }
        if (join < 0) return fail(REWL_ERR_STATE, "windows %d and %d have no common joining bin", a, a + 1);
        offset[(size_t)a + 1] = (pa[join - lo_a] + offset[(size_t)a]) - pb[join - lo_b];
        cut[(size_t)a] = join;
        last = join;
    }
    for (int b = 0; b < nb; ++b) out[b] = -INFINITY;
    for (int a = 0; a < h; ++a) {
        const int lo = e_lo[(size_t)a] + 2 * N;
        const int first = a == 0 ? lo : cut[(size_t)a - 1] + 1;
        const int end = a == h - 1 ? lo + W : cut[(size_t)a];
        for (int b = first; b <= end; ++b)
            if (mw[(size_t)a * B + (b - lo)]) out[b] = lw[(size_t)a * B + (b - lo)] + offset[(size_t)a];
    }
    return REWL_OK;
}

// Shift so that sum over visited bins of g(E) = q^N.
void normalise_total(int q, int N, double *v, int nb) {
    double top = -INFINITY;
    for (int b = 0; b < nb; ++b) top = v[b] > top ? v[b] : top;
    if (top == -INFINITY) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b)
        if (v[b] != -INFINITY) s += std::exp(v[b] - top);
    const double shift = (double)N * std::log((double)q) - (top + std::log(s));
    for (int b = 0; b < nb; ++b)
        if (v[b] != -INFINITY) v[b] += shift;
}

}  // namespace host
}  // namespace rewl

using rewl::host::join_windows;
using rewl::host::normalise_total;

namespace {

uint64_t fnv1a(const unsigned char *p, size_t n, uint64_t hsh = 1469598103934665603ull) {
    for (size_t i = 0; i < n; ++i) {
        hsh ^= p[i];
        hsh *= 1099511628211ull;
    }
    return hsh;
}

bool same_params(const rewl_params &a, const rewl_params &b) {
    return a.q == b.q && a.L == b.L && a.h == b.h && a.overlap == b.overlap && a.m == b.m &&
           a.lnf_final == b.lnf_final && a.flatness == b.flatness && a.exchange_interval == b.exchange_interval &&
           a.seed == b.seed;
}

struct SaveHeader {
    char magic[8];
    uint32_t version;
    uint32_t spin_bits;
    uint32_t schedule;
    uint32_t pad;
    rewl_params prm;
    uint64_t payload;
    uint64_t checksum;
};

}  // namespace


namespace rewl {
namespace host {

namespace {
struct Allocator {
    void *(*alloc)(size_t bytes, void *ctx) = nullptr;  // nullptr: cudaMalloc
    void (*free)(void *ptr, void *ctx) = nullptr;
    void *ctx = nullptr;
};
Allocator g_alloc;
}  // namespace

cudaError_t dev_alloc(DevBlock &b, size_t bytes) {
    b = DevBlock{};
    if (!g_alloc.alloc) return cudaMalloc(&b.ptr, bytes);
    void *p = g_alloc.alloc(bytes, g_alloc.ctx);
    if (!p) return cudaErrorMemoryAllocation;
    b.ptr = p;
    b.hooked = true;
    b.free_fn = g_alloc.free;
    b.ctx = g_alloc.ctx;
    if (((uintptr_t)p & 255u) != 0) {  // the state parts are laid out at 256-byte offsets
        dev_free(b);
        return cudaErrorMemoryAllocation;
    }
    return cudaSuccess;
}

void dev_free(DevBlock &b) {
    if (!b.ptr) return;
    if (!b.hooked) cudaFree(b.ptr);
    else if (b.free_fn) b.free_fn(b.ptr, b.ctx);  // (an allocator without a free keeps its memory)
    b = DevBlock{};
}

void set_allocator(void *(*alloc)(size_t, void *), void (*free_fn)(void *, void *), void *ctx) {
    g_alloc.alloc = alloc;
    g_alloc.free = alloc ? free_fn : nullptr;
    g_alloc.ctx = alloc ? ctx : nullptr;
}

rewl_status prepare_instance(rewl_s *h, const rewl_params &p, int spin_bits, int lanes, int spin_capacity_bits) {
    rewl_status st = check_params(p, spin_bits);
    if (st) return st;
    std::vector<int32_t> e_lo;
    int W = 0;
    if (!window_geometry(p.L, p.h, p.overlap, e_lo, W))
        return fail(REWL_ERR_ARG, "window width below 8 bins (L=%d, h=%d, overlap=%g)", p.L, p.h, p.overlap);
    h->prm = p;
    h->e_lo = e_lo;
    Model &M = h->M;
    M.q = p.q;
    M.L = p.L;
    M.N = p.L * p.L;
    M.W = W;
    M.B = W + 1;
    M.h = p.h;
    M.m = p.m;
    M.G = p.h * p.m;
    M.bits = spin_bits ? spin_bits : (p.q <= 16 ? 4 : 8);
    M.wpc = (M.N * M.bits + 31) / 32;
    M.key0 = (uint32_t)(p.seed & 0xffffffffull);
    M.key1 = (uint32_t)(p.seed >> 32);
    M.divL = (uint32_t)((0x100000000ull + (unsigned long long)p.L - 1) / (unsigned long long)p.L);
    M.K = p.exchange_interval;
    M.lnf_final = p.lnf_final;
    M.flatness = p.flatness;
    M.schedule = rewl::SCHED_HALVING;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) return fail(REWL_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    h->plan = rewl::plan_sweep(M, h->sms, (size_t)h->smem_optin, rewl::SWEEP_FAST, lanes);
    if (h->plan.P < 1)
        return fail(REWL_ERR_ARG, "one walker needs %zu bytes of shared memory (> %d)",
                    rewl::fast_smem_per_walker(M, h->plan.lanes, h->plan.lat_global != 0), h->smem_optin);
    const size_t G = (size_t)M.G, B = (size_t)M.B, hh = (size_t)M.h;
    const int cap_bits = spin_capacity_bits > M.bits ? spin_capacity_bits : M.bits;
    const size_t wpc_cap = (size_t)((M.N * cap_bits + 31) / 32);
    const size_t sizes[] = {G * wpc_cap * 4, G * 4, G * 4, G * 8, G * B * 8, G * B * 4, hh * B, hh * 4, hh * 8, hh * 4, hh,
                            G, G * 4, G * (B + 2 * rewl::kShadowPad) * 8, hh, (size_t)rewl::kTieLog * 16,
                            sizeof(Ctl)};
    size_t off = 0;
    h->parts.clear();
    for (size_t sz : sizes) {
        h->parts.push_back({off, sz});
        off += align256(sz);
    }
    h->dbytes = off;
    return REWL_OK;
}

void carve_instance(rewl_s *h, void *base) {
    h->dmem = base;
    auto at = [&](int i) { return (void *)((char *)base + h->parts[(size_t)i].off); };
    State &S = h->S;
    S.spins = (uint32_t *)at(0);
    S.cfg_E = (int32_t *)at(1);
    S.slot_cfg = (uint32_t *)at(2);
    S.t = (unsigned long long *)at(3);
    S.lng = (double *)at(4);
    S.H = (uint32_t *)at(5);
    S.mask = (uint8_t *)at(6);
    S.e_lo = (int32_t *)at(7);
    S.lnf = (double *)at(8);
    S.iter = (int32_t *)at(9);
    S.done = (uint8_t *)at(10);
    S.rt_end = (uint8_t *)at(11);
    S.rt_trips = (uint32_t *)at(12);
    S.shadow = (long long *)at(13);
    S.phase = (uint8_t *)at(14);
    S.tlog = (unsigned long long *)at(15);
    S.ctl = (Ctl *)at(16);  // last: save / load treat the last part as the control block
}

cudaError_t init_instance_async(rewl_s *h, cudaStream_t s) {
    const size_t hh = (size_t)h->M.h;
    std::vector<double> lnf0(hh, 1.0);  // ln f_0 = 1
    cudaError_t e = cudaMemsetAsync(h->dmem, 0, h->dbytes, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->S.e_lo, h->e_lo.data(), hh * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->S.lnf, lnf0.data(), hh * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // lnf0 lives on this stack frame
    if (e == cudaSuccess) e = rewl::launch_init(h->M, h->S, s);
    return e;
}

rewl_status read_status(rewl_s *h) { return read_ctl(h); }

}  // namespace host
}  // namespace rewl

// ============================================================================
extern "C" {

const char *rewl_last_error(void) { return g_last_error.c_str(); }

const char *rewl_version(void) { return "rewl-gb300 0.1 (sm_103a)"; }

rewl_status rewl_create_ext(const rewl_params *prm, int spin_bits, rewl_t *out) {
    REWL_API_TRY
    const rewl::host::Range range("rewl_create");
    if (!prm || !out) return fail(REWL_ERR_ARG, "NULL argument");
    *out = nullptr;
    rewl_s *h = new rewl_s();
    auto cleanup = [&](rewl_status s) {
        rewl_destroy(h);
        return s;
    };
    rewl_status st = rewl::host::prepare_instance(h, *prm, spin_bits, 0);
    if (st) return cleanup(st);
    cudaError_t e = rewl::host::dev_alloc(h->dblock, h->dbytes);
    if (e != cudaSuccess)
        return cleanup(fail(REWL_ERR_NOMEM, "device memory (%zu bytes): %s", h->dbytes, cudaGetErrorString(e)));
    rewl::host::carve_instance(h, h->dblock.ptr);
    e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(fail(REWL_ERR_CUDA, "stream: %s", cudaGetErrorString(e)));
    h->stream = h->own_stream;
    e = cudaMallocHost(&h->h_ctl, sizeof(Ctl));
    if (e != cudaSuccess) return cleanup(fail(REWL_ERR_NOMEM, "cudaMallocHost: %s", cudaGetErrorString(e)));
    e = rewl::host::init_instance_async(h, h->stream);
    if (e == cudaSuccess) e = rewl::prepare_sweep(h->M, h->plan);
    if (e != cudaSuccess) return cleanup(fail(REWL_ERR_CUDA, "initialisation: %s", cudaGetErrorString(e)));
    st = read_ctl(h);
    if (st) return cleanup(st);
    st = build_graph(h);
    if (st) return cleanup(st);
    *out = h;
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_create(int q, int L, int h, double overlap, int m, double lnf_final, double flatness,
                        long long exchange_interval, unsigned long long seed, rewl_t *out) {
    REWL_API_TRY
    rewl_params p;
    p.q = q;
    p.L = L;
    p.h = h;
    p.overlap = overlap;
    p.m = m;
    p.lnf_final = lnf_final;
    p.flatness = flatness;
    p.exchange_interval = exchange_interval;
    p.seed = seed;
    return rewl_create_ext(&p, 0, out);
    REWL_API_CATCH
}

void rewl_set_allocator(void *(*alloc)(size_t bytes, void *ctx), void (*free_fn)(void *ptr, void *ctx), void *ctx) {
    rewl::host::set_allocator(alloc, free_fn, ctx);
}

void rewl_destroy(rewl_t h) {
    if (!h || !h->owns) return;  // instances of a batch belong to the batch
    if (h->stream) cudaStreamSynchronize(h->stream);
    rewl::host::dev_free(h->prod_block);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    if (h->h_ctl) cudaFreeHost(h->h_ctl);
    rewl::host::dev_free(h->dblock);
    delete h;
}

rewl_status rewl_set_stream(rewl_t h, void *stream) {
    REWL_API_TRY
    if (h && !h->owns) return fail(REWL_ERR_STATE, "this instance belongs to a batch: run the batch");
    if (!h) return fail(REWL_ERR_ARG, "NULL handle");
    REWL_CUDA(cudaStreamSynchronize(h->stream));
    h->stream = stream ? (cudaStream_t)stream : h->own_stream;
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_run_async(rewl_t h, long long rounds) {
    REWL_API_TRY
    if (h && !h->owns) return fail(REWL_ERR_STATE, "this instance belongs to a batch: run the batch");
    if (!h) return fail(REWL_ERR_ARG, "NULL handle");
    if (h->M.production) return fail(REWL_ERR_STATE, "in production: use rewl_production_run");
    if (rounds < 0) return fail(REWL_ERR_ARG, "rounds < 0");
    return enqueue_rounds(h, rounds);
    REWL_API_CATCH
}

rewl_status rewl_run_phase(rewl_t h, int phase) {
    REWL_API_TRY
    const rewl::host::Range range(phase == REWL_PHASE_SWEEP ? "rewl_phase_sweep"
                                  : phase == REWL_PHASE_CHECK ? "rewl_phase_check"
                                                              : "rewl_phase_exchange");
    if (h && !h->owns) return fail(REWL_ERR_STATE, "this instance belongs to a batch: run the batch");
    if (!h) return fail(REWL_ERR_ARG, "NULL handle");
    if (h->M.production) return fail(REWL_ERR_STATE, "in production: use rewl_production_run");
    switch (phase) {
    case REWL_PHASE_SWEEP: REWL_CUDA(rewl::launch_sweep(h->M, h->S, h->plan, h->stream)); break;
    case REWL_PHASE_CHECK: REWL_CUDA(rewl::launch_window_check(h->M, h->S, h->stream)); break;
    case REWL_PHASE_EXCHANGE: REWL_CUDA(rewl::launch_exchange(h->M, h->S, h->stream)); break;
    default: return fail(REWL_ERR_ARG, "unknown phase %d", phase);
    }
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_set_option(rewl_t h, int option, long long value) {
    REWL_API_TRY
    if (h && !h->owns) return fail(REWL_ERR_STATE, "this instance belongs to a batch: run the batch");
    if (!h) return fail(REWL_ERR_ARG, "NULL handle");
    if (h->M.production) return fail(REWL_ERR_STATE, "in production: options are fixed");
    int kind = h->plan.kind, lanes = h->plan.lanes, lat_mode = h->lat_mode;
    if (option == REWL_OPT_STALL_MS) {  // host side only: no re-plan
        if (value < 0) return fail(REWL_ERR_ARG, "stall limit %lld ms < 0", value);
        h->stall_ms = value;
        return REWL_OK;
    }
    int schedule = h->M.schedule;
    if (option == REWL_OPT_SCHEDULE) {
        if (value != rewl::SCHED_HALVING && value != rewl::SCHED_INV_T)
            return fail(REWL_ERR_ARG, "ln f schedule %lld not 0 or 1", value);
        schedule = (int)value;
    } else if (option == REWL_OPT_SWEEP_KERNEL) {
        if (value != 0 && value != 1) return fail(REWL_ERR_ARG, "sweep kernel %lld not 0 or 1", value);
        kind = value == 0 ? rewl::SWEEP_FAST : rewl::SWEEP_REFERENCE;
        lanes = 0;
    } else if (option == REWL_OPT_LANES) {
        if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8 && value != 16 && value != 32)
            return fail(REWL_ERR_ARG, "lanes per walker %lld not 0, 1, 2, 4, 8, 16 or 32", value);
        lanes = (int)value;
    } else if (option == REWL_OPT_LATTICE) {
        if (value < 0 || value > 2) return fail(REWL_ERR_ARG, "lattice placement %lld not 0, 1 or 2", value);
        lat_mode = (int)value;
    } else {
        return fail(REWL_ERR_ARG, "unknown option %d", option);
    }
    const rewl::SweepPlan plan = rewl::plan_sweep(h->M, h->sms, (size_t)h->smem_optin, kind, lanes, lat_mode);
    if (plan.P < 1) return fail(REWL_ERR_ARG, "configuration does not fit in shared memory");
    REWL_CUDA(cudaStreamSynchronize(h->stream));
    REWL_CUDA(rewl::prepare_sweep(h->M, plan));
    h->plan = plan;
    h->lat_mode = lat_mode;
    h->M.schedule = schedule;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    return build_graph(h);
    REWL_API_CATCH
}

rewl_status rewl_autotune(rewl_t h, int rounds, rewl_tune_entry *entries, int max_entries, int *n_entries) {
    REWL_API_TRY
    const rewl::host::Range range("rewl_autotune");
    if (h && !h->owns) return fail(REWL_ERR_STATE, "this instance belongs to a batch: tune the batch");
    if (!h) return fail(REWL_ERR_ARG, "NULL handle");
    if (h->M.production) return fail(REWL_ERR_STATE, "in production: options are fixed");
    if (max_entries < 0 || (max_entries > 0 && !entries)) return fail(REWL_ERR_ARG, "entries");
    if (rounds <= 0) rounds = 2;
    if (n_entries) *n_entries = 0;
    if (h->plan.kind != rewl::SWEEP_FAST) return REWL_OK;  // the reference sweep has nothing to tune
    cudaEvent_t e0, e1;
    REWL_CUDA(cudaEventCreate(&e0));
    REWL_CUDA(cudaEventCreate(&e1));
    int best = 0, n_done = 0;
    double best_rate = -1.0;
    rewl_status st = REWL_OK;
    for (int lanes : {32, 16, 8, 4, 2, 1}) {
        st = rewl_set_option(h, REWL_OPT_LANES, lanes);
        if (st == REWL_ERR_ARG) {  // does not fit in shared memory: not a candidate
            st = REWL_OK;
            continue;
        }
        if (st) break;
        st = enqueue_rounds(h, 1);  // settles the new plan
        if (st == REWL_OK) st = read_ctl(h);
        if (st || h->h_ctl->all_done) break;
        const unsigned long long f0 = h->h_ctl->flips;
        cudaError_t e = cudaEventRecord(e0, h->stream);
        if (e == cudaSuccess) st = enqueue_rounds(h, rounds);
        if (e == cudaSuccess && st == REWL_OK) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess && st == REWL_OK) st = read_ctl(h);
        float ms = 0.0f;
        if (e == cudaSuccess && st == REWL_OK) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess && st == REWL_OK) st = fail(REWL_ERR_CUDA, "autotune timing: %s", cudaGetErrorString(e));
        if (st) break;
        const double rate = ms > 0.0f ? (double)(h->h_ctl->flips - f0) / (ms * 1e-3) : 0.0;
        if (n_done < max_entries) {
            rewl_tune_entry &en = entries[n_done];
            en.spin_bits = h->M.bits;
            en.lanes = lanes;
            en.cta_kb = (int)(h->plan.smem / 1024);
            en.threads = h->plan.threads;
            en.flips_per_s = rate;
        }
        ++n_done;
        if (rate > best_rate) {
            best_rate = rate;
            best = lanes;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    if (n_entries) *n_entries = std::min(n_done, max_entries);
    return best_rate >= 0.0 ? rewl_set_option(h, REWL_OPT_LANES, best) : REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_get_option(rewl_t h, int option, long long *value) {
    REWL_API_TRY
    if (!h || !value) return fail(REWL_ERR_ARG, "NULL argument");
    if (option == REWL_OPT_SWEEP_KERNEL) *value = h->plan.kind == rewl::SWEEP_FAST ? 0 : 1;
    else if (option == REWL_OPT_LANES) *value = h->plan.lanes;
    else if (option == REWL_OPT_WALKERS_PER_CTA) *value = h->plan.P;
    else if (option == REWL_OPT_LATTICE) *value = h->plan.lat_global;
    else if (option == REWL_OPT_STALL_MS) *value = h->stall_ms;
    else if (option == REWL_OPT_SCHEDULE) *value = h->M.schedule;
    else return fail(REWL_ERR_ARG, "unknown option %d", option);
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_sync(rewl_t h, int *converged) {
    REWL_API_TRY
    if (!h) return fail(REWL_ERR_ARG, "NULL handle");
    rewl_status st = read_ctl(h);
    if (converged) *converged = h->h_ctl->all_done ? 1 : 0;
    return st;
    REWL_API_CATCH
}

rewl_status rewl_run(rewl_t h, long long max_rounds, int *converged) {
    REWL_API_TRY
    const rewl::host::Range range("rewl_run");
    if (h && !h->owns) return fail(REWL_ERR_STATE, "this instance belongs to a batch: run the batch");
    if (!h) return fail(REWL_ERR_ARG, "NULL handle");
    if (h->M.production) return fail(REWL_ERR_STATE, "in production: use rewl_production_run");
    long long left = max_rounds;
    rewl_status st = read_ctl(h);
    // stall watchdog: progress = iterations completed over all windows; a
    // window that follows ln f = 1/t lowers ln f every round, so it progresses
    std::vector<int32_t> iters(h->stall_ms > 0 ? (size_t)h->M.h : 0);
    std::vector<uint8_t> phase(h->stall_ms > 0 ? (size_t)h->M.h : 0), done(phase.size());
    long long progress = -1;
    auto t_progress = std::chrono::steady_clock::now();
    while (st == REWL_OK && !h->h_ctl->all_done && (max_rounds <= 0 || left > 0)) {
        const long long n = (max_rounds <= 0 || left >= kGraphRounds) ? kGraphRounds : left;
        st = enqueue_rounds(h, n);
        if (st == REWL_OK) st = read_ctl(h);
        left -= n;
        if (st == REWL_OK && h->stall_ms > 0 && !h->h_ctl->all_done) {
            REWL_CUDA(cudaMemcpy(iters.data(), h->S.iter, iters.size() * 4, cudaMemcpyDeviceToHost));
            long long sum = 0;
            for (int32_t v : iters) sum += v;
            bool moving = false;
            if (h->M.schedule == rewl::SCHED_INV_T) {
                REWL_CUDA(cudaMemcpy(phase.data(), h->S.phase, phase.size(), cudaMemcpyDeviceToHost));
                REWL_CUDA(cudaMemcpy(done.data(), h->S.done, done.size(), cudaMemcpyDeviceToHost));
                for (size_t w = 0; w < phase.size(); ++w) moving = moving || (phase[w] && !done[w]);
            }
            const auto now = std::chrono::steady_clock::now();
            if (sum != progress || moving) {
                progress = sum;
                t_progress = now;
            } else if (std::chrono::duration_cast<std::chrono::milliseconds>(now - t_progress).count() > h->stall_ms) {
                st = fail(REWL_ERR_TIMEOUT, "no window finished an iteration for %lld ms (round %llu)", h->stall_ms,
                          (unsigned long long)h->h_ctl->round);
            }
        }
    }
    if (converged) *converged = h->h_ctl->all_done ? 1 : 0;
    return st;
    REWL_API_CATCH
}

rewl_status rewl_get_window_lng(rewl_t h, int w, double *out, size_t len, int *e_lo) {
    REWL_API_TRY
    if (!h || !out) return fail(REWL_ERR_ARG, "NULL argument");
    if (w < 0 || w >= h->M.h) return fail(REWL_ERR_ARG, "window %d outside [0, %d)", w, h->M.h);
    if (len != (size_t)h->M.B) return fail(REWL_ERR_ARG, "len %zu != W + 1 = %d", len, h->M.B);
    REWL_CUDA(cudaMemcpyAsync(out, h->S.lng + (size_t)w * h->M.m * h->M.B, len * 8, cudaMemcpyDeviceToHost, h->stream));
    REWL_CUDA(cudaStreamSynchronize(h->stream));
    if (e_lo) *e_lo = h->e_lo[(size_t)w];
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_get_lng(rewl_t h, double *out, size_t len, int partial) {
    REWL_API_TRY
    if (!h || !out) return fail(REWL_ERR_ARG, "NULL argument");
    const Model &M = h->M;
    if (len != (size_t)(2 * M.N + 1)) return fail(REWL_ERR_ARG, "len %zu != 2N + 1 = %d", len, 2 * M.N + 1);
    rewl_status st = read_ctl(h);
    if (st) return st;
    if (!partial && !h->h_ctl->all_done) return fail(REWL_ERR_STATE, "run has not converged");
    std::vector<double> lw((size_t)M.h * M.B);
    std::vector<uint8_t> mw((size_t)M.h * M.B);
    // walker 0 of every window: rows w*m of the [G][B] ln g array
    REWL_CUDA(cudaMemcpy2DAsync(lw.data(), (size_t)M.B * 8, h->S.lng, (size_t)M.m * M.B * 8, (size_t)M.B * 8, (size_t)M.h,
                                cudaMemcpyDeviceToHost, h->stream));
    REWL_CUDA(cudaMemcpyAsync(mw.data(), h->S.mask, mw.size(), cudaMemcpyDeviceToHost, h->stream));
    REWL_CUDA(cudaStreamSynchronize(h->stream));
    st = join_windows(M.N, M.W, h->e_lo, lw, mw, out);
    if (st) return st;
    normalise_total(M.q, M.N, out, 2 * M.N + 1);
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_get_info(rewl_t h, rewl_info *info) {
    REWL_API_TRY
    if (!h || !info) return fail(REWL_ERR_ARG, "NULL argument");
    info->N = h->M.N;
    info->W = h->M.W;
    info->walkers = h->M.G;
    info->spin_bits = h->M.bits;
    info->device_bytes = h->dbytes;
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_get_stats(rewl_t h, rewl_stats *s) {
    REWL_API_TRY
    if (!h || !s) return fail(REWL_ERR_ARG, "NULL argument");
    std::vector<double> lnf((size_t)h->M.h);
    std::vector<uint8_t> done((size_t)h->M.h);
    REWL_CUDA(cudaMemcpyAsync(lnf.data(), h->S.lnf, lnf.size() * 8, cudaMemcpyDeviceToHost, h->stream));
    REWL_CUDA(cudaMemcpyAsync(done.data(), h->S.done, done.size(), cudaMemcpyDeviceToHost, h->stream));
    rewl_status st = read_ctl(h);
    const Ctl &c = *h->h_ctl;
    s->rounds = (long long)c.round;
    s->flips = (long long)c.flips;
    s->accepted = (long long)c.accepted;
    s->exch_tried = (long long)c.xtried;
    s->exch_accepted = (long long)c.xacc;
    s->near_ties = (long long)c.ties;
    s->slow_decisions = (long long)c.slow;
    s->seq_steps = (long long)c.seq;
    s->windows_done = 0;
    s->min_lnf = INFINITY;
    s->max_lnf = -INFINITY;
    for (size_t i = 0; i < done.size(); ++i) {
        s->windows_done += done[i] ? 1 : 0;
        s->min_lnf = std::min(s->min_lnf, lnf[i]);
        s->max_lnf = std::max(s->max_lnf, lnf[i]);
    }
    s->converged = c.all_done ? 1 : 0;
    return st;
    REWL_API_CATCH
}

static rewl_status field_geometry(rewl_t h, int field, void **dev, size_t *bytes) {
    const size_t G = (size_t)h->M.G, B = (size_t)h->M.B, hh = (size_t)h->M.h;
    switch (field) {
    case REWL_FIELD_SPINS: *dev = nullptr; *bytes = G * (size_t)h->M.N; break;
    case REWL_FIELD_ENERGY: *dev = nullptr; *bytes = G * 4; break;
    case REWL_FIELD_REPLICA: *dev = h->S.slot_cfg; *bytes = G * 4; break;
    case REWL_FIELD_STEPS: *dev = h->S.t; *bytes = G * 8; break;
    case REWL_FIELD_LNG: *dev = h->S.lng; *bytes = G * B * 8; break;
    case REWL_FIELD_HIST: *dev = h->S.H; *bytes = G * B * 4; break;
    case REWL_FIELD_MASK: *dev = h->S.mask; *bytes = hh * B; break;
    case REWL_FIELD_LNF: *dev = h->S.lnf; *bytes = hh * 8; break;
    case REWL_FIELD_ITER: *dev = h->S.iter; *bytes = hh * 4; break;
    case REWL_FIELD_DONE: *dev = h->S.done; *bytes = hh; break;
    case REWL_FIELD_ELO: *dev = h->S.e_lo; *bytes = hh * 4; break;
    case REWL_FIELD_ROUND: *dev = &h->S.ctl->round; *bytes = 8; break;
    case REWL_FIELD_TRIPS: *dev = h->S.rt_trips; *bytes = G * 4; break;
    case REWL_FIELD_TRIP_END: *dev = h->S.rt_end; *bytes = G; break;
    case REWL_FIELD_PHASE: *dev = h->S.phase; *bytes = hh; break;
    case REWL_FIELD_TIES: *dev = h->S.tlog; *bytes = (size_t)rewl::kTieLog * 16; break;
    default: return fail(REWL_ERR_ARG, "unknown field %d", field);
    }
    return REWL_OK;
}

rewl_status rewl_get_field(rewl_t h, int field, void *out, size_t bytes) {
    REWL_API_TRY
    if (!h || !out) return fail(REWL_ERR_ARG, "NULL argument");
    void *dev;
    size_t need;
    rewl_status st = field_geometry(h, field, &dev, &need);
    if (st) return st;
    if (bytes != need) return fail(REWL_ERR_ARG, "field %d needs %zu bytes, got %zu", field, need, bytes);
    if (field == REWL_FIELD_SPINS) {
        uint8_t *tmp = nullptr;
        REWL_CUDA(cudaMallocAsync((void **)&tmp, need, h->stream));
        cudaError_t e = rewl::launch_get_spins(h->M, h->S, tmp, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, need, cudaMemcpyDeviceToHost, h->stream);
        cudaFreeAsync(tmp, h->stream);
        if (e != cudaSuccess) return fail(REWL_ERR_CUDA, "spins: %s", cudaGetErrorString(e));
    } else if (field == REWL_FIELD_ENERGY) {
        std::vector<uint32_t> slot((size_t)h->M.G);
        std::vector<int32_t> cfgE((size_t)h->M.G);
        REWL_CUDA(cudaMemcpyAsync(slot.data(), h->S.slot_cfg, slot.size() * 4, cudaMemcpyDeviceToHost, h->stream));
        REWL_CUDA(cudaMemcpyAsync(cfgE.data(), h->S.cfg_E, cfgE.size() * 4, cudaMemcpyDeviceToHost, h->stream));
        REWL_CUDA(cudaStreamSynchronize(h->stream));
        int32_t *o = (int32_t *)out;
        for (size_t g = 0; g < slot.size(); ++g) o[g] = cfgE[slot[g]];
        return REWL_OK;
    } else {
        REWL_CUDA(cudaMemcpyAsync(out, dev, need, cudaMemcpyDeviceToHost, h->stream));
    }
    REWL_CUDA(cudaStreamSynchronize(h->stream));
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_set_field(rewl_t h, int field, const void *in, size_t bytes) {
    REWL_API_TRY
    if (!h || !in) return fail(REWL_ERR_ARG, "NULL argument");
    if (field == REWL_FIELD_ELO || field == REWL_FIELD_REPLICA || field == REWL_FIELD_ENERGY ||
        field == REWL_FIELD_TIES)
        return fail(REWL_ERR_ARG, "field %d is read-only", field);
    void *dev;
    size_t need;
    rewl_status st = field_geometry(h, field, &dev, &need);
    if (st) return st;
    if (bytes != need) return fail(REWL_ERR_ARG, "field %d needs %zu bytes, got %zu", field, need, bytes);
    if (field == REWL_FIELD_SPINS) {
        const uint8_t *s = (const uint8_t *)in;
        for (size_t i = 0; i < need; ++i)
            if (s[i] >= h->M.q) return fail(REWL_ERR_ARG, "spin value %d >= q", (int)s[i]);
        uint8_t *tmp = nullptr;
        REWL_CUDA(cudaMallocAsync((void **)&tmp, need, h->stream));
        cudaError_t e = cudaMemcpyAsync(tmp, in, need, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = rewl::launch_set_spins(h->M, h->S, tmp, h->stream);
        cudaFreeAsync(tmp, h->stream);
        if (e != cudaSuccess) return fail(REWL_ERR_CUDA, "spins: %s", cudaGetErrorString(e));
    } else {
        REWL_CUDA(cudaMemcpyAsync(dev, in, need, cudaMemcpyHostToDevice, h->stream));
    }
    REWL_CUDA(cudaStreamSynchronize(h->stream));
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_save(rewl_t h, void *buf, size_t *len) {
    REWL_API_TRY
    if (!h || !len) return fail(REWL_ERR_ARG, "NULL argument");
    if (h->M.production) return fail(REWL_ERR_STATE, "in production: checkpoints hold WL runs only");
    size_t payload = 0;
    for (auto &p : h->parts) payload += p.bytes;
    const size_t need = sizeof(SaveHeader) + payload;
    if (!buf) {
        *len = need;
        return REWL_OK;
    }
    if (*len < need) return fail(REWL_ERR_ARG, "buffer of %zu bytes < %zu", *len, need);
    unsigned char *dst = (unsigned char *)buf + sizeof(SaveHeader);
    for (size_t i = 0; i < h->parts.size(); ++i) {
        const auto &p = h->parts[i];
        const void *src = i + 1 == h->parts.size() ? (const void *)h->S.ctl : (const void *)((char *)h->dmem + p.off);
        REWL_CUDA(cudaMemcpyAsync(dst, src, p.bytes, cudaMemcpyDeviceToHost, h->stream));
        dst += p.bytes;
    }
    REWL_CUDA(cudaStreamSynchronize(h->stream));
    SaveHeader hd;
    std::memset(&hd, 0, sizeof hd);
    std::memcpy(hd.magic, "REWLSAV1", 8);
    hd.version = 2;
    hd.spin_bits = (uint32_t)h->M.bits;
    hd.schedule = (uint32_t)h->M.schedule;
    hd.prm = h->prm;
    hd.payload = payload;
    hd.checksum = fnv1a((const unsigned char *)buf + sizeof(SaveHeader), payload);
    std::memcpy(buf, &hd, sizeof hd);
    *len = need;
    return REWL_OK;
    REWL_API_CATCH
}

rewl_status rewl_load(rewl_t h, const void *buf, size_t len) {
    REWL_API_TRY
    if (!h || !buf) return fail(REWL_ERR_ARG, "NULL argument");
    if (h->M.production) return fail(REWL_ERR_STATE, "in production: checkpoints hold WL runs only");
    if (len < sizeof(SaveHeader)) return fail(REWL_ERR_ARG, "blob too short");
    SaveHeader hd;
    std::memcpy(&hd, buf, sizeof hd);
    size_t payload = 0;
    for (auto &p : h->parts) payload += p.bytes;
    if (std::memcmp(hd.magic, "REWLSAV1", 8) != 0 || hd.version != 2) return fail(REWL_ERR_ARG, "not a rewl state blob");
    if (hd.payload != payload || len != sizeof(SaveHeader) + payload || hd.spin_bits != (uint32_t)h->M.bits ||
        !same_params(hd.prm, h->prm))
        return fail(REWL_ERR_ARG, "blob belongs to an instance with other parameters");
    if (hd.schedule != (uint32_t)h->M.schedule)
        return fail(REWL_ERR_ARG, "blob was saved under ln f schedule %u, the handle runs %d", hd.schedule,
                    h->M.schedule);
    if (fnv1a((const unsigned char *)buf + sizeof(SaveHeader), payload) != hd.checksum)
        return fail(REWL_ERR_ARG, "blob checksum mismatch (corrupted)");
    const unsigned char *src = (const unsigned char *)buf + sizeof(SaveHeader);
    for (size_t i = 0; i < h->parts.size(); ++i) {
        const auto &p = h->parts[i];
        void *dst = i + 1 == h->parts.size() ? (void *)h->S.ctl : (void *)((char *)h->dmem + p.off);
        REWL_CUDA(cudaMemcpyAsync(dst, src, p.bytes, cudaMemcpyHostToDevice, h->stream));
        src += p.bytes;
    }
    REWL_CUDA(cudaStreamSynchronize(h->stream));
    return read_ctl(h);
    REWL_API_CATCH
}

}  // extern "C"
