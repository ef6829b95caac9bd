// api_host.cpp -- cmm_multiply_host: the whole path on host buffers, with the
// operand copies and the copy-back of the estimate overlapped with the
// computation on an internal copy stream per device.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "api_common.h"

using namespace cmm;
using namespace cmm::api;

namespace {

// ---- the host-buffer path: copies overlapped with the computation ----------
// The inner index is split in up to four parts when the operands are large:
// part c + 1 is copied to the device on an internal copy stream while part c
// is prepared and sketched on the caller's stream.  The estimate is extracted
// in row blocks, each copied back while the next is extracted.
constexpr int kHostRowBlocks = 8;   // at most; one per 16 MiB of the estimate

// operands of 64 MiB or more: two parts; 256 MiB or more: three; 1 GiB or
// more: four (every part at least 512 inner indices)
int host_parts(int64_t m, int64_t k, int64_t p, size_t es) {
    const double bytes = (double)(m + p) * (double)k * (double)es;
    if (k < 512 || bytes < 64.0 * 1048576.0) return 1;
    if (bytes >= 1024.0 * 1048576.0 && k >= 4 * 512) return 4;
    return bytes >= 256.0 * 1048576.0 && k >= 3 * 512 ? 3 : 2;
}

// Ratio of the parts' sizes along the inner index: while part c is sketched
// part c + 1 is copied, so neither waits when part c + 1 is `ratio` times part
// c, ratio = sketch time / copy time per inner index.  Per inner index the
// copy moves (m + p) elements over the host link (~211 GB/s measured on this
// GPU's host path) and the sketch does d (2 b log2 b + b) butterfly
// operations (~18 Tops/s FP32, ~13 Tops/s BF16 blocks, ~6 Tops/s exact fixed
// point, ~0.45 Tops/s FP64).
// Kept within [1/2, 3]: only the first part's copy is exposed, and it shrinks
// as the later parts grow.
double host_part_ratio(int64_t m, int64_t p, int d, int L, size_t es, int prec) {
    const double b = std::ldexp(1.0, L);
    const double copy_t = (double)(m + p) * (double)es / 211e9;
    const double rate = prec == CMM_PREC_F64    ? 0.45e12
                        : prec == CMM_PREC_FX64 ? 6e12
                        : prec_tc(prec)         ? 13e12
                                                : 18e12;
    const double sketch_t = (double)d * (2.0 * b * L + b) / rate;
    return std::min(3.0, std::max(0.5, sketch_t / copy_t));
}

// row blocks of the estimate: one per 16 MiB (at most kHostRowBlocks, at
// least 256 rows each), so that only the last block's copy is left exposed
int host_row_blocks(int64_t m, int64_t p) {
    const double bytes = (double)m * (double)p * 8.0;
    int nrb = (int)std::min<double>(kHostRowBlocks, std::floor(bytes / (16.0 * 1048576.0)));
    while (nrb > 1 && m < (int64_t)nrb * 256) --nrb;
    return std::max(1, nrb);
}

size_t host_sketch_ws(int64_t m, int64_t k, int64_t p, int d, int L, int dtype, int prec,
                      int transA) {
    SketchPlan pl;
    if (!plan_sketch(m, k, p, d, L, dtype, prec, transA, transA ? m : k, p, pl,
                     host_parts(m, k, p, dtype_size(dtype)),
                     host_part_ratio(m, p, d, L, dtype_size(dtype), prec)))
        return 0;
    return pl.total;
}

// per device: one copy stream and its events, created on first use; a call
// holds the device's mutex for its whole duration (calls from several host
// threads on one device run one after the other)
constexpr int kMaxDevices = 64;
constexpr int kCopyEvents = 4 + kMaxParts + kHostRowBlocks;
struct CopyCtx {
    std::mutex mu;
    bool ready = false;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev[kCopyEvents] = {};
};
CopyCtx g_copy[kMaxDevices];

int copy_ctx(CopyCtx *&out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(CMM_ERR_RANGE, "device index %d out of range", dev);
    out = &g_copy[dev];
    return CMM_OK;
}

int copy_ctx_init(CopyCtx &c) {
    if (c.ready) return CMM_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&c.cs, cudaStreamNonBlocking);
    for (int i = 0; e == cudaSuccess && i < kCopyEvents; ++i)
        e = cudaEventCreateWithFlags(&c.ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "copy stream set-up");
    c.ready = true;
    return CMM_OK;
}

}  // namespace

extern "C" {

size_t cmm_multiply_host_workspace_bytes(int64_t m, int64_t k, int64_t p, int32_t d,
                                         int32_t log2b, int32_t dtype, int32_t prec,
                                         int32_t transA, int64_t capacity) {
    const size_t mw = cmm_multiply_workspace_bytes(m, k, p, d, log2b, dtype, prec, transA);
    if (!mw || capacity < 0) return 0;
    const size_t sk = host_sketch_ws(m, k, p, d, log2b, dtype, prec, transA);
    const size_t ex = extract_ws_bytes(m, p, d);
    const size_t es = dtype_size(dtype);
    return align_up((size_t)m * k * es) + align_up((size_t)k * p * es) +
           align_up((size_t)m * p * sizeof(double)) +
           align_up((size_t)capacity * (2 * sizeof(int32_t) + sizeof(double))) +
           align_up((size_t)d * (size_t(1) << log2b) * sizeof(double)) + std::max(sk, ex);
}

int cmm_multiply_host(const void *A, int64_t lda, int32_t transA, const void *B, int64_t ldb,
                      int32_t dtype, int64_t m, int64_t k, int64_t p, const cmm_hashes *hs,
                      int32_t prec, int32_t reduce, double *C, int64_t ldc, double tau,
                      int64_t capacity, int32_t *I, int32_t *J, double *V, int64_t *count,
                      void *ws, size_t ws_bytes, void *stream) {
    g_err.clear();
    int rc = check_hashes(hs);
    if (rc) return rc;
    rc = check_operands(A, lda, transA, B, ldb, dtype, m, k, p, prec);
    if (rc) return rc;
    rc = check_prec_sizes(prec, hs->log2b, m, p);
    if (rc) return rc;
    if (reduce != CMM_MEDIAN && reduce != CMM_MEAN) return fail(CMM_ERR_ARG, "bad reduce %d", reduce);
    if (C && ldc < p) return fail(CMM_ERR_ARG, "ldc = %lld < p", (long long)ldc);
    if (count && capacity < 0) return fail(CMM_ERR_ARG, "negative capacity");
    if (count && capacity > 0 && (!I || !J || !V)) return fail(CMM_ERR_ARG, "I, J or V is NULL");
    const int64_t cap = count ? capacity : 0;
    if (count) *count = 0;
    const HhRange hr = hh_range(tau);
    const size_t need = cmm_multiply_host_workspace_bytes(m, k, p, hs->d, hs->log2b, dtype, prec,
                                                          transA, cap);
    rc = check_ws(ws, ws_bytes, need);
    if (rc) return rc;
    CopyCtx *cx = nullptr;
    rc = copy_ctx(cx);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(cx->mu);
    rc = copy_ctx_init(*cx);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaStream_t cs = cx->cs;
    cudaEvent_t ev_start = cx->ev[0], ev_done = cx->ev[1];
    cudaEvent_t *ev_in = cx->ev + 4, *ev_out = cx->ev + 4 + kMaxParts;
    const size_t es = dtype_size(dtype);
    char *base = static_cast<char *>(ws);
    char *dA = base;
    base += align_up((size_t)m * k * es);
    char *dB = base;
    base += align_up((size_t)k * p * es);
    double *dC = reinterpret_cast<double *>(base);
    base += align_up((size_t)m * p * sizeof(double));
    int32_t *dI = reinterpret_cast<int32_t *>(base);
    int32_t *dJ = dI + cap;
    double *dV = reinterpret_cast<double *>(base + align_up((size_t)cap * 2 * sizeof(int32_t)));
    base += align_up((size_t)cap * (2 * sizeof(int32_t) + sizeof(double)));
    const size_t rbytes = align_up((size_t)hs->d * (size_t(1) << hs->log2b) * sizeof(double));
    double *Rw = reinterpret_cast<double *>(base);
    void *scratch = base + rbytes;

    // the copy stream starts after the work already queued on the caller's stream
    cudaError_t e = cudaEventRecord(ev_start, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_start, 0);
    if (e != cudaSuccess) return cuda_fail(e, "copy stream ordering");
    // operands, part by part (A as stored: m x k, or k x m when transA; the
    // device copy is compact)
    SketchPlan pl;
    const int nparts = host_parts(m, k, p, es);
    const double ratio = host_part_ratio(m, p, hs->d, hs->log2b, es, prec);
    plan_sketch(m, k, p, hs->d, hs->log2b, dtype, prec, transA, transA ? m : k, p, pl, nparts,
                ratio);
    const int64_t acols = transA ? m : k;
    for (int c = 0; c < pl.nparts; ++c) {
        const int64_t k0 = pl.kb[c], kp = pl.kb[c + 1] - pl.kb[c];
        if (m > 0 && kp > 0) {
            Span sp("h2d_A", cs, 0);
            if (transA)
                e = cudaMemcpy2DAsync(dA + k0 * m * es, m * es, static_cast<const char *>(A) + k0 * lda * es,
                                      lda * es, m * es, kp, cudaMemcpyHostToDevice, cs);
            else
                e = cudaMemcpy2DAsync(dA + k0 * es, k * es, static_cast<const char *>(A) + k0 * es,
                                      lda * es, kp * es, m, cudaMemcpyHostToDevice, cs);
            if (e != cudaSuccess) return cuda_fail(e, "copy A to device");
        }
        if (kp > 0 && p > 0) {
            Span sp("h2d_B", cs, 0);
            e = cudaMemcpy2DAsync(dB + k0 * p * es, p * es, static_cast<const char *>(B) + k0 * ldb * es,
                                  ldb * es, p * es, kp, cudaMemcpyHostToDevice, cs);
            if (e != cudaSuccess) return cuda_fail(e, "copy B to device");
        }
        e = cudaEventRecord(ev_in[c], cs);
        if (e != cudaSuccess) return cuda_fail(e, "operand part event");
    }
    // the same split as the copies above (run_sketch plans with the same arguments)
    rc = run_sketch(dA, acols > 0 ? acols : 1, transA, dB, p > 0 ? p : 1, dtype, m, k, p, hs,
                    prec, Rw, scratch, s, pl.nparts, ev_in, ratio);
    if (rc) return rc;
    // the estimate in row blocks, each copied back while the next is extracted
    if (m > 0 && p > 0) {
        HashParams hp;
        fill_params(hs, hp);
        ExtractWs ew = carve_extract(scratch, m, p, hs->d);
        {
            Span sp("hash_tables", s);
            e = launch_hash_tables(hp, hs->d, hs->log2b, m, p, ew.H1, ew.H2, s);
        }
        if (e == cudaSuccess && count)
            e = cudaMemsetAsync(ew.ncand, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) return cuda_fail(e, "hash tables");
        const int nrb = host_row_blocks(m, p);
        for (int i = 0; i < nrb; ++i) {
            const int64_t i0 = m * i / nrb, mb = m * (i + 1) / nrb - i0;
            if (mb == 0) continue;
            {
                Span sp("extract", s);
                e = count ? launch_hh_cand(Rw, ew.H1 + i0, ew.H2, hs->d, hs->log2b, mb, p, m, i0,
                                           reduce, hr, dC + i0 * p, p, ew.tcounts + i0 * ew.nt,
                                           ew.tsrc + i0 * ew.nt, ew.nt, ew.ncand, ew.ccap, ew.CI,
                                           ew.CJ, ew.CV, s)
                          : launch_extract(Rw, ew.H1 + i0, ew.H2, hs->d, hs->log2b, mb, p,
                                           reduce, dC + i0 * p, p, m, s);
            }
            if (e != cudaSuccess) return cuda_fail(e, "extract kernel");
            if (C) {
                e = cudaEventRecord(ev_out[i], s);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_out[i], 0);
                if (e != cudaSuccess) return cuda_fail(e, "row block event");
                Span sp("d2h_C", cs, 0);
                e = cudaMemcpy2DAsync(C + i0 * ldc, ldc * sizeof(double), dC + i0 * p,
                                      p * sizeof(double), p * sizeof(double), mb,
                                      cudaMemcpyDeviceToHost, cs);
                if (e != cudaSuccess) return cuda_fail(e, "copy C to host");
            }
        }
    }
    int hh_rc = CMM_OK;
    if (count && m > 0 && p > 0) {
        hh_rc = finish_hh(carve_extract(scratch, m, p, hs->d), true, dC, p, m, p, hr, dI, dJ, dV,
                          cap, count, s);
        if (hh_rc != CMM_OK && hh_rc != CMM_ERR_CAPACITY) return hh_rc;
        const int64_t n = std::min(*count, cap);
        if (n > 0) {
            Span sp("d2h_hh", s, 0);
            e = cudaMemcpyAsync(I, dI, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(J, dJ, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(V, dV, n * sizeof(double), cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return cuda_fail(e, "copy heavy hitters to host");
        }
    }
    // the caller's stream ends after the last copy
    e = cudaEventRecord(ev_done, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_done, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "multiply_host sync");
    if (hh_rc == CMM_ERR_CAPACITY)
        return fail(CMM_ERR_CAPACITY, "%lld heavy hitters, capacity %lld", (long long)*count,
                    (long long)cap);
    return CMM_OK;
}

}  // extern "C"
