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

// One cached lookup per device: the array's device address and the id of the
// context it was looked up in.  Context ids are never reused within a process,
// so after a cudaDeviceReset (which destroys the primary context) or under
// another context on the same device the id differs and the lookup runs again.
struct Cached {
    void *addr = nullptr;
    unsigned long long ctx_id = 0;
    bool valid = false;
};
Cached g_cache[kMaxDevices];

// driver entry points reached through the runtime (no link-time libcuda)
typedef int (*ctx_get_current_fn)(void **);
typedef int (*ctx_get_id_fn)(void *, unsigned long long *);

// id of the calling thread's current context; false when it cannot be read
// (then the address is looked up again on every call)
bool current_context_id(unsigned long long *id) {
    static ctx_get_current_fn get_current = nullptr;
    static ctx_get_id_fn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<ctx_get_current_fn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<ctx_get_id_fn>(f);
        cudaGetLastError();
    });
    if (!get_current || !get_id) return false;
    void *ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) return false;
    return get_id(ctx, id) == 0;
}

// Device address of the scratch array in the current device's context.  In
// host code the array's name is only a host-side stand-in; a kernel must get
// the address cudaGetSymbolAddress returns.  It is looked up with the device
// current on the first call in each context and kept for that context.
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
    // initialises the device's primary context if no context is current yet
    // (so that the id below names the context the lookup and the launches use)
    e = cudaSetDevice(dev);
    if (e != cudaSuccess) {
        char msg[256];
        std::snprintf(msg, sizeof msg, "cmm_sketch_noalloc: context set-up: %s", cudaGetErrorString(e));
        return cmm::set_error(CMM_ERR_CUDA, msg);
    }
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    std::lock_guard<std::mutex> lk(g_mu);
    Cached &c = g_cache[dev];
    if (!(have_id && c.valid && c.ctx_id == id)) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sketch_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char msg[256];
            std::snprintf(msg, sizeof msg, "cmm_sketch_noalloc: cudaGetSymbolAddress: %s",
                          cudaGetErrorString(e));
            c.valid = false;
            return cmm::set_error(CMM_ERR_CUDA, msg);
        }
        c.addr = p;
        c.ctx_id = id;
        c.valid = have_id;
    }
    *out = c.addr;
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
