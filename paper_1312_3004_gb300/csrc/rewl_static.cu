// rewl_static.cu -- rewl_run_static: a whole REWL run whose working state lives
// in a fixed, file-scope device array instead of memory allocated per call.
//
// Who needs it: callers that cannot call cudaMalloc.  Examples are code that
// runs under a framework whose caching allocator owns the device memory and
// forbids raw allocations, a process whose device-memory budget is fixed when
// it starts, and latency-critical loops that cannot afford the implicit device
// synchronisation of cudaMalloc / cudaFree while other streams are busy.  Such
// a caller passes its inputs (the parameters) and its outputs (device buffers
// it already owns); this entry point allocates nothing.
//
// The array g_rewl_static_scratch (kStaticScratchBytes) is reserved on every
// GPU that loads the library and is kept until the process exits.  Every call
// on a device shares it: the state of the previous call stays in it, so each
// call clears what must start at zero, and calls whose work overlaps on the
// GPU (two host threads, or two streams) race on it.
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include <cuda.h>

#include "rewl.h"
#include "rewl_host_internal.hpp"
#include "rewl_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_rewl_static_scratch[kStaticScratchBytes];

// Where the array lives on each device, and in which context that address was
// looked up: a context torn down (cudaDeviceReset, the primary context released)
// unloads the module, and the next context maps the array somewhere else.
struct ScratchAddr {
    void *ctx = nullptr;
    unsigned char *addr = nullptr;
};
std::mutex g_setup_mu;
ScratchAddr g_scratch[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
CtxGetCurrentFn g_ctx_get_current = nullptr;

// The driver's cuCtxGetCurrent, reached through the runtime (no link to libcuda).
rewl_status current_context(void **ctx) {
    if (!g_ctx_get_current) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return rewl::host::fail(REWL_ERR_CUDA, "cuCtxGetCurrent not available: %s", cudaGetErrorString(e));
        g_ctx_get_current = (CtxGetCurrentFn)fn;
    }
    CUcontext c = nullptr;
    if (g_ctx_get_current(&c) != CUDA_SUCCESS) return rewl::host::fail(REWL_ERR_CUDA, "cuCtxGetCurrent failed");
    *ctx = (void *)c;
    return REWL_OK;
}

// The device address of the array.  In host code the symbol name is only a
// host-side stand-in, so the address is looked up with the device current
// (cudaGetSymbolAddress, which also creates the context) and cached per
// device; a cached address is used only in the context it was looked up in.
rewl_status scratch_on_current_device(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return rewl::host::fail(REWL_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return rewl::host::fail(REWL_ERR_ARG, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_setup_mu);
    void *ctx = nullptr;
    rewl_status st = current_context(&ctx);
    if (st) return st;
    ScratchAddr &a = g_scratch[dev];
    if (!a.addr || !ctx || a.ctx != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_rewl_static_scratch);
        if (e != cudaSuccess)
            return rewl::host::fail(REWL_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        st = current_context(&ctx);  // the lookup made the context current if there was none
        if (st) return st;
        a.ctx = ctx;
        a.addr = (unsigned char *)p;
    }
    *out = a.addr;
    return REWL_OK;
}

}  // namespace

extern "C" rewl_status rewl_run_static(const rewl_params *prm, int spin_bits, long long max_rounds,
                                       double *lng_out, unsigned char *mask_out, size_t out_bins,
                                       int *converged, void *stream) {
    REWL_API_TRY
    if (!prm || !lng_out) return rewl::host::fail(REWL_ERR_ARG, "NULL argument");
    // The same checks, window table, model, sweep plan and array layout as
    // rewl_create_ext, so that a static run and an allocating run are one run.
    rewl_s inst;
    rewl_s *h = &inst;
    rewl_status st = rewl::host::prepare_instance(h, *prm, spin_bits, 0);
    if (st) return st;
    const rewl::Model &M = h->M;
    const size_t B = (size_t)M.B, hh = (size_t)M.h;
    if (out_bins != hh * B)
        return rewl::host::fail(REWL_ERR_ARG, "out_bins %zu != h * (W + 1) = %zu", out_bins, hh * B);
    if (h->dbytes > kStaticScratchBytes)
        return rewl::host::fail(REWL_ERR_ARG, "instance needs %zu bytes of state; the static scratch holds %zu",
                                h->dbytes, kStaticScratchBytes);

    unsigned char *base = nullptr;
    st = scratch_on_current_device(&base);
    if (st) return st;
    rewl::host::carve_instance(h, base);
    const rewl::State &S = h->S;
    const rewl::SweepPlan &plan = h->plan;

    cudaStream_t s = (cudaStream_t)stream;
    rewl::Ctl ctl{};
    auto read_ctl = [&]() -> rewl_status {
        cudaError_t e2 = cudaMemcpyAsync(&ctl, S.ctl, sizeof ctl, cudaMemcpyDeviceToHost, s);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
        if (e2 != cudaSuccess) return rewl::host::fail(REWL_ERR_CUDA, "status read: %s", cudaGetErrorString(e2));
        if (ctl.error & rewl::ERR_OVERFLOW) return rewl::host::fail(REWL_ERR_OVERFLOW, "a histogram bin reached 2^31");
        if (ctl.error & rewl::ERR_ENTRY) return rewl::host::fail(REWL_ERR_STATE, "a walker could not enter its window");
        if (ctl.error & rewl::ERR_BOUNDS)
            return rewl::host::fail(REWL_ERR_STATE, "an index failed its bounds check (debug build)");
        if (ctl.error & rewl::ERR_ENERGY)
            return rewl::host::fail(REWL_ERR_STATE, "a walker's energy differs from its recount (debug build)");
        return REWL_OK;
    };

    // everything the previous call left behind is cleared
    // (zeroing, the window table, ln f = 1, the initial configurations: the
    // same set-up as rewl_create_ext, into the array)
    cudaError_t e = rewl::host::init_instance_async(h, s);
    if (e == cudaSuccess) e = rewl::prepare_sweep(M, plan);
    if (e != cudaSuccess) return rewl::host::fail(REWL_ERR_CUDA, "initialisation: %s", cudaGetErrorString(e));
    st = read_ctl();
    if (st) return st;

    long long done_rounds = 0;
    while (!ctl.all_done && (max_rounds <= 0 || done_rounds < max_rounds)) {
        long long n = 8;
        if (max_rounds > 0 && max_rounds - done_rounds < n) n = max_rounds - done_rounds;
        for (long long r = 0; r < n && e == cudaSuccess; ++r) {
            e = rewl::launch_sweep(M, S, plan, s);
            if (e == cudaSuccess) e = rewl::launch_window_check(M, S, s);
            if (e == cudaSuccess) e = rewl::launch_exchange(M, S, s);
        }
        if (e != cudaSuccess) return rewl::host::fail(REWL_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
        done_rounds += n;
        st = read_ctl();
        if (st) return st;
    }

    // walker 0 of every window: rows w*m of the [G][B] ln g array
    e = cudaMemcpy2DAsync(lng_out, B * 8, S.lng, (size_t)M.m * B * 8, B * 8, hh, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && mask_out) e = cudaMemcpyAsync(mask_out, S.mask, hh * B, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return rewl::host::fail(REWL_ERR_CUDA, "result copy: %s", cudaGetErrorString(e));
    if (converged) *converged = ctl.all_done ? 1 : 0;
    return REWL_OK;
    REWL_API_CATCH
}
