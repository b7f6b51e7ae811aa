// rewl_host_internal.hpp -- host-side instance record shared by the
// single-instance driver (rewl_host.cu) and the batch engine (rewl_batch.cu).
#pragma once
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "rewl.h"
#include "rewl_internal.cuh"

// Every entry point of the C ABI returns a status and lets no C++ exception
// (a failed host allocation inside a standard container) cross the ABI.
#define REWL_API_TRY try {
#define REWL_API_CATCH                                                                     \
    }                                                                                      \
    catch (const std::bad_alloc &) {                                                       \
        return rewl::host::fail(REWL_ERR_NOMEM, "host memory exhausted");                  \
    }                                                                                      \
    catch (...) {                                                                          \
        return rewl::host::fail(REWL_ERR_STATE, "unexpected host error");                 \
    }

namespace rewl {
namespace host {

// Device memory of a handle, a batch or a server: from the allocator set with
// rewl_set_allocator (else cudaMalloc), returned through the matching free.
struct DevBlock {
    void *ptr = nullptr;
    bool hooked = false;                              // false: cudaMalloc / cudaFree
    void (*free_fn)(void *ptr, void *ctx) = nullptr;  // hooked: nullptr means kept by the allocator
    void *ctx = nullptr;
};
// cudaSuccess, or cudaErrorMemoryAllocation (also for memory not 256-byte aligned).
cudaError_t dev_alloc(DevBlock &b, size_t bytes);
void dev_free(DevBlock &b);
void set_allocator(void *(*alloc)(size_t, void *), void (*free_fn)(void *, void *), void *ctx);

// A named range on the host timeline of a profiler (NVTX; free when none is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};
}  // namespace host
}  // namespace rewl

struct rewl_s {
    rewl_params prm{};
    rewl::Model M{};
    rewl::State S{};
    rewl::SweepPlan plan{};
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    void *dmem = nullptr;  // base of this instance's device arrays
    rewl::host::DevBlock dblock;  // the allocation behind dmem (stand-alone handles)
    size_t dbytes = 0;
    rewl::Ctl *h_ctl = nullptr;  // pinned mirror of the device control block
    std::vector<int32_t> e_lo;
    cudaGraphExec_t graph = nullptr;
    int sms = 0, smem_optin = 0;
    int lat_mode = 0;  // REWL_OPT_LATTICE: 0 by size, 1 global memory, 2 shared memory
    long long stall_ms = 0;  // REWL_OPT_STALL_MS: rewl_run gives up after this long without progress
    // byte offsets of the state arrays relative to dmem (for save / load); the
    // last part is the control block
    struct Part { size_t off, bytes; };
    std::vector<Part> parts;
    // false for an instance that lives inside a batch: the batch owns its
    // memory, stream and pinned status block, and runs its rounds
    bool owns = true;
    // fixed-weight production (rewl_production_start): H(E, O) and spin counts
    rewl::host::DevBlock prod_block;
};

namespace rewl {
namespace host {


// Checks the parameters, computes the window table and the sizes of the device
// arrays (h->parts, h->dbytes) and plans the sweep.  lanes: lanes per walker of
// the fast sweep (0 = from the walker count).  spin_capacity_bits (0 = the
// packing chosen): the configuration buffers are sized for this packing, so
// that a batch can repack its spins in place.  No device memory is touched.
rewl_status prepare_instance(rewl_s *h, const rewl_params &p, int spin_bits, int lanes, int spin_capacity_bits = 0);
// Points h->S at the arrays of a region of h->dbytes bytes at `base`.
void carve_instance(rewl_s *h, void *base);
// Queues zeroing, the window table, ln f = 1 and the initial configurations.
cudaError_t init_instance_async(rewl_s *h, cudaStream_t s);
// Reads the control block (synchronises h->stream) and maps its error bits.
rewl_status read_status(rewl_s *h);
rewl_status fail(rewl_status st, const char *fmt, ...);
// Joins h window pieces (lw, mw: h x (W + 1), window-major) into out[2N + 1]
// (Sec. 2, Fig. 2): each neighbouring pair meets at the bin of their overlap
// where the pieces' slopes d ln g / dE differ least; -inf where no window
// visited a bin.  REWL_ERR_STATE when a pair has no usable bin.
rewl_status join_windows(int N, int W, const std::vector<int32_t> &e_lo, const std::vector<double> &lw,
                         const std::vector<uint8_t> &mw, double *out);
// Shifts the finite entries of v[nb] so that sum g = q^N.
void normalise_total(int q, int N, double *v, int nb);

}  // namespace host
}  // namespace rewl
