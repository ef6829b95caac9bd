// noalloc.cu -- cmm_sketch_noalloc: the sketch for callers that cannot
// allocate device memory.
//
// Some callers have no way to hand the library a workspace: a serving process
// that reserved its whole device-memory budget at start-up and forbids further
// cudaMalloc calls, a plugin whose host application owns every device
// allocation, or a latency-critical path that cannot afford cudaMalloc's
// implicit device-wide synchronisation.  This entry point needs no workspace:
// its scratch (the converted operands when a conversion is needed, the
// per-block partial sums and the reduced sums before the inverse transform)
// lives in the file-scope device array below, of CMM_SKETCH_NOALLOC_SCRATCH_BYTES.
// Every GPU that loads the library holds that array until the process exits.
//
// All calls share the one array, and it keeps whatever the previous call left
// in it.  Nothing in it has to start at zero: the sketch kernel writes every
// partial sum it later reads and the finish pass writes every reduced sum.
// Calls that overlap on the GPU (two streams, or two host threads) race on the
// array and give wrong results; serialise them.
#include <cstdio>
#include <mutex>

#include "cmm_internal.h"

static __device__ __align__(256) unsigned char g_sketch_noalloc_scratch[CMM_SKETCH_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 256;
std::mutex g_mu;
void *g_scratch[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device.  In host code the array's name is only a host-side stand-in; a
// kernel must get the address cudaGetSymbolAddress returns.
int scratch_on_current_device(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        char msg[256];
        std::snprintf(msg, sizeof msg, "cmm_sketch_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
        return cmm::set_error(CMM_ERR_CUDA, msg);
    }
    if (dev < 0 || dev >= kMaxDevices)
        return cmm::set_error(CMM_ERR_RANGE, "cmm_sketch_noalloc: device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sketch_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char msg[256];
            std::snprintf(msg, sizeof msg, "cmm_sketch_noalloc: cudaGetSymbolAddress: %s",
                          cudaGetErrorString(e));
            return cmm::set_error(CMM_ERR_CUDA, msg);
        }
        g_scratch[dev] = p;
    }
    *out = g_scratch[dev];
    return CMM_OK;
}

}  // namespace

extern "C" int cmm_sketch_noalloc(const void *A, int64_t lda, int32_t transA, const void *B,
                                  int64_t ldb, int32_t dtype, int64_t m, int64_t k, int64_t p,
                                  const cmm_hashes *hs, int32_t prec, double *R, void *stream) {
    if (!hs) return cmm::set_error(CMM_ERR_ARG, "hashes: null pointer");
    // the size check needs no GPU and comes first
    // (invalid sizes give 0 here and are reported by cmm_sketch's own checks)
    const size_t need = cmm_sketch_workspace_bytes(m, k, p, hs->d, hs->log2b, dtype, prec, transA);
    if (need > CMM_SKETCH_NOALLOC_SCRATCH_BYTES) {
        char msg[256];
        std::snprintf(msg, sizeof msg,
                      "cmm_sketch_noalloc: this problem needs %zu bytes of scratch, more than the "
                      "%zu-byte static array; use cmm_sketch with a workspace",
                      need, (size_t)CMM_SKETCH_NOALLOC_SCRATCH_BYTES);
        return cmm::set_error(CMM_ERR_RANGE, msg);
    }
    void *scratch = nullptr;
    int rc = scratch_on_current_device(&scratch);
    if (rc != CMM_OK) return rc;
    return cmm_sketch(A, lda, transA, B, ldb, dtype, m, k, p, hs, prec, R, scratch,
                      CMM_SKETCH_NOALLOC_SCRATCH_BYTES, stream);
}
