// rewl_production.cu -- fixed-weight production runs behind include/rewl.h:
// once the density of states is estimated, configurations are sampled with
// the fixed weights 1/g(E) and distributions H(E, O) of an observable
// recorded (Sec. 3.2 of arXiv:1312.3004 does this for its lipid model).
// Here O is the Potts majority count; each window keeps its walkers' ln g and
// ln f = 0; a production round is K steps of every walker of every window
// (production_kernel, rewl_kernels.cu) followed by a replica exchange between
// every pair (a, a + 1), a = round (mod 2), with Eq. 1, which keeps the
// fixed-weight ensembles of neighbouring windows in detailed balance.
#include "rewl.h"
#include "rewl_host_internal.hpp"

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

#define PROD_CUDA(call)                                                                          \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return rewl::host::fail(REWL_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

extern "C" {

rewl_status rewl_production_start(rewl_t h, int n_obins) {
    REWL_API_TRY
    if (h && !h->owns) return rewl::host::fail(REWL_ERR_STATE, "this instance belongs to a batch");
    if (!h) return rewl::host::fail(REWL_ERR_ARG, "NULL handle");
    rewl::Model &M = h->M;
    const int qlo = (M.N + M.q - 1) / M.q;
    if (n_obins < 1 || n_obins > M.N - qlo + 1)
        return rewl::host::fail(REWL_ERR_ARG, "n_obins %d outside [1, N - ceil(N/q) + 1 = %d]", n_obins,
                                M.N - qlo + 1);
    rewl_status st = rewl::host::read_status(h);  // also waits for queued rounds
    if (st) return st;
    const size_t heo_bytes = (size_t)M.h * M.B * (size_t)n_obins * 8, cnt_bytes = (size_t)M.G * M.q * 4;
    rewl::host::dev_free(h->prod_block);
    h->S.heo = nullptr;
    h->S.cnt = nullptr;
    cudaError_t e = rewl::host::dev_alloc(h->prod_block, align256(heo_bytes) + cnt_bytes);
    if (e != cudaSuccess)
        return rewl::host::fail(REWL_ERR_NOMEM, "production histogram (%zu bytes): %s", heo_bytes,
                                cudaGetErrorString(e));
    h->S.heo = (unsigned long long *)h->prod_block.ptr;
    h->S.cnt = (int32_t *)((char *)h->prod_block.ptr + align256(heo_bytes));
    PROD_CUDA(cudaMemsetAsync(h->S.heo, 0, heo_bytes, h->stream));
    PROD_CUDA(cudaMemsetAsync(h->S.lnf, 0, (size_t)M.h * 8, h->stream));  // ln f = 0 (+0.0 is all zero bits)
    PROD_CUDA(cudaMemsetAsync(h->S.H, 0, (size_t)M.G * M.B * 4, h->stream));
    M.production = 1;
    M.n_obins = n_obins;
    PROD_CUDA(rewl::launch_count_spins(M, h->S, h->stream));
    return rewl::host::read_status(h);
    REWL_API_CATCH
}

rewl_status rewl_production_run(rewl_t h, long long rounds) {
    REWL_API_TRY
    const rewl::host::Range range("rewl_production_run");
    if (h && !h->owns) return rewl::host::fail(REWL_ERR_STATE, "this instance belongs to a batch");
    if (!h) return rewl::host::fail(REWL_ERR_ARG, "NULL handle");
    if (!h->M.production) return rewl::host::fail(REWL_ERR_STATE, "no production started (rewl_production_start)");
    if (rounds < 0) return rewl::host::fail(REWL_ERR_ARG, "rounds < 0");
    for (long long r = 0; r < rounds; ++r) {
        PROD_CUDA(rewl::launch_production_sweep(h->M, h->S, h->stream));
        PROD_CUDA(rewl::launch_exchange(h->M, h->S, h->stream));
        if ((r & 63) == 63) {
            rewl_status st = rewl::host::read_status(h);
            if (st) return st;
        }
    }
    return rewl::host::read_status(h);
    REWL_API_CATCH
}

rewl_status rewl_production_histogram(rewl_t h, unsigned long long *out, size_t len) {
    REWL_API_TRY
    if (!h || !out) return rewl::host::fail(REWL_ERR_ARG, "NULL argument");
    if (!h->M.production) return rewl::host::fail(REWL_ERR_STATE, "no production started (rewl_production_start)");
    const size_t need = (size_t)h->M.h * h->M.B * (size_t)h->M.n_obins;
    if (len != need) return rewl::host::fail(REWL_ERR_ARG, "len %zu != h * (W + 1) * n_obins = %zu", len, need);
    PROD_CUDA(cudaMemcpyAsync(out, h->S.heo, need * 8, cudaMemcpyDeviceToHost, h->stream));
    PROD_CUDA(cudaStreamSynchronize(h->stream));
    return REWL_OK;
    REWL_API_CATCH
}

}  // extern "C"
