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
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "rewl.h"
#include "rewl_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_rewl_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};

rewl_status fail_static(rewl_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    rewl::set_error(buf);
    return st;
}

// The device address of the array.  In host code the symbol name is only a
// host-side stand-in, so the address is looked up once per device, with that
// device current, and cached.
rewl_status scratch_on_current_device(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_static(REWL_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail_static(REWL_ERR_ARG, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_rewl_static_scratch);
        if (e != cudaSuccess)
            return fail_static(REWL_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = (unsigned char *)p;
    }
    *out = g_scratch_addr[dev];
    return REWL_OK;
}

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

// Window start energies and ln f = 1 for every window, written on the device so
// that the host needs no buffer of its own.
__global__ void static_setup_kernel(int32_t *e_lo, double *lnf, int h, int N, int W) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= h) return;
    const long long R = 2LL * N;
    const long long off = h > 1 ? (2LL * i * (R - W) + (h - 1)) / (2LL * (h - 1)) : 0LL;
    e_lo[i] = (int32_t)(-2LL * N + off);
    lnf[i] = 1.0;
}

}  // namespace

extern "C" rewl_status rewl_run_static(const rewl_params *prm, int spin_bits, long long max_rounds,
                                       double *lng_out, unsigned char *mask_out, size_t out_bins,
                                       int *converged, void *stream) {
    if (!prm || !lng_out) return fail_static(REWL_ERR_ARG, "NULL argument");
    const rewl_params &p = *prm;
    if (p.q < 2 || p.q > 255 || p.L < 3 || p.L > 1024 || p.h < 1 || p.m < 1 || p.m > 256 ||
        !(p.overlap >= 0.0 && p.overlap < 1.0) || !(p.lnf_final > 0.0 && p.lnf_final < 1.0) ||
        !(p.flatness > 0.0 && p.flatness < 1.0) || p.exchange_interval < 1 ||
        (spin_bits != 0 && spin_bits != 4 && spin_bits != 8) || (spin_bits == 4 && p.q > 16))
        return fail_static(REWL_ERR_ARG, "parameter out of range");
    const long long N = (long long)p.L * p.L, R = 2 * N;
    long long W = (long long)std::ceil((double)R / (1.0 + (double)(p.h - 1) * (1.0 - p.overlap)));
    if (W > R) W = R;
    if (W < 8) return fail_static(REWL_ERR_ARG, "window width below 8 bins");

    rewl::Model M{};
    M.q = p.q;
    M.L = p.L;
    M.N = (int)N;
    M.W = (int)W;
    M.B = (int)W + 1;
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
    const size_t G = (size_t)M.G, B = (size_t)M.B, hh = (size_t)M.h;
    if (out_bins != hh * B) return fail_static(REWL_ERR_ARG, "out_bins %zu != h * (W + 1) = %zu", out_bins, hh * B);

    const size_t sizes[16] = {G * M.wpc * 4, G * 4, G * 4, G * 8, G * B * 8, G * B * 4,
                              hh * B, hh * 4, hh * 8, hh * 4, hh, G, G * 4, G * (B + 2 * rewl::kShadowPad) * 8,
                              hh, sizeof(rewl::Ctl)};
    size_t offs[16], total = 0;
    for (int i = 0; i < 16; ++i) {
        offs[i] = total;
        total += round256(sizes[i]);
    }
    if (total > kStaticScratchBytes)
        return fail_static(REWL_ERR_ARG, "instance needs %zu bytes of state; the static scratch holds %zu", total,
                           kStaticScratchBytes);

    unsigned char *base = nullptr;
    rewl_status st = scratch_on_current_device(&base);
    if (st) return st;
    int dev = 0, sms = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);

    rewl::State S{};
    S.spins = (uint32_t *)(base + offs[0]);
    S.cfg_E = (int32_t *)(base + offs[1]);
    S.slot_cfg = (uint32_t *)(base + offs[2]);
    S.t = (unsigned long long *)(base + offs[3]);
    S.lng = (double *)(base + offs[4]);
    S.H = (uint32_t *)(base + offs[5]);
    S.mask = (uint8_t *)(base + offs[6]);
    S.e_lo = (int32_t *)(base + offs[7]);
    S.lnf = (double *)(base + offs[8]);
    S.iter = (int32_t *)(base + offs[9]);
    S.done = (uint8_t *)(base + offs[10]);
    S.rt_end = (uint8_t *)(base + offs[11]);
    S.rt_trips = (uint32_t *)(base + offs[12]);
    S.shadow = (long long *)(base + offs[13]);
    S.phase = (uint8_t *)(base + offs[14]);
    S.ctl = (rewl::Ctl *)(base + offs[15]);

    cudaStream_t s = (cudaStream_t)stream;
    const rewl::SweepPlan plan = rewl::plan_sweep(M, sms, (size_t)optin);
    if (plan.P < 1) return fail_static(REWL_ERR_ARG, "lattice too large for shared memory");
    rewl::Ctl ctl{};
    auto read_ctl = [&]() -> rewl_status {
        cudaError_t e2 = cudaMemcpyAsync(&ctl, S.ctl, sizeof ctl, cudaMemcpyDeviceToHost, s);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
        if (e2 != cudaSuccess) return fail_static(REWL_ERR_CUDA, "status read: %s", cudaGetErrorString(e2));
        if (ctl.error & rewl::ERR_OVERFLOW) return fail_static(REWL_ERR_OVERFLOW, "a histogram bin reached 2^31");
        if (ctl.error & rewl::ERR_ENTRY) return fail_static(REWL_ERR_STATE, "a walker could not enter its window");
        if (ctl.error & rewl::ERR_BOUNDS) return fail_static(REWL_ERR_STATE, "an index failed its bounds check (debug build)");
        if (ctl.error & rewl::ERR_ENERGY)
            return fail_static(REWL_ERR_STATE, "a walker's energy differs from its recount (debug build)");
        return REWL_OK;
    };

    // everything the previous call left behind is cleared
    cudaError_t e = cudaMemsetAsync(base, 0, total, s);
    if (e == cudaSuccess) {
        static_setup_kernel<<<(M.h + 127) / 128, 128, 0, s>>>(S.e_lo, S.lnf, M.h, M.N, M.W);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = rewl::launch_init(M, S, s);
    if (e == cudaSuccess) e = rewl::prepare_sweep(M, plan);
    if (e != cudaSuccess) return fail_static(REWL_ERR_CUDA, "initialisation: %s", cudaGetErrorString(e));
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
        if (e != cudaSuccess) return fail_static(REWL_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
        done_rounds += n;
        st = read_ctl();
        if (st) return st;
    }

    // walker 0 of every window: rows w*m of the [G][B] ln g array
    e = cudaMemcpy2DAsync(lng_out, B * 8, S.lng, (size_t)M.m * B * 8, B * 8, hh, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && mask_out) e = cudaMemcpyAsync(mask_out, S.mask, hh * B, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_static(REWL_ERR_CUDA, "result copy: %s", cudaGetErrorString(e));
    if (converged) *converged = ctl.all_done ? 1 : 0;
    return REWL_OK;
}
