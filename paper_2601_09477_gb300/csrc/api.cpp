// api.cpp -- the C ABI of libcmm (include/cmm.h), core entry points: error
// text and tracing, hash parameters, Compress, Decompress, the heavy-hitter
// lists and the device-buffer multiply.
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

// splitmix64 (Steele, Lea & Flood 2014): state += golden gamma, then mix
uint64_t splitmix64(uint64_t &state) {
    state += 0x9e3779b97f4a7c15ULL;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" {

const char *cmm_last_error(void) { return g_err.c_str(); }

const char *cmm_version(void) { return "cmm 0.1.0 (sm_103a)"; }

int cmm_trace_enable(int32_t on) {
    g_err.clear();
    std::lock_guard<std::mutex> lk(g_tr_mu);
    if (on) {
        for (auto &r : g_tr) {
            g_ev_pool.push_back(r.a);
            g_ev_pool.push_back(r.b);
        }
        g_tr.clear();
    }
    g_tr_on = on != 0;
    return CMM_OK;
}

int cmm_trace_read(int32_t max_entries, char *names, int64_t *launches, double *total_ms,
                   int32_t *n_out) {
    g_err.clear();
    if (!n_out || (max_entries > 0 && (!names || !launches || !total_ms)))
        return fail(CMM_ERR_ARG, "null pointer");
    std::lock_guard<std::mutex> lk(g_tr_mu);
    std::vector<std::string> keys;
    std::vector<int64_t> cnt;
    std::vector<double> tot;
    for (auto &r : g_tr) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return cuda_fail(e, "trace event");
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) return cuda_fail(e, "trace elapsed");
        size_t q = 0;
        while (q < keys.size() && keys[q] != r.name) ++q;
        if (q == keys.size()) {
            keys.push_back(r.name);
            cnt.push_back(0);
            tot.push_back(0.0);
        }
        cnt[q] += r.launches;
        tot[q] += ms;
    }
    const int n = (int)keys.size();
    for (int q = 0; q < n && q < max_entries; ++q) {
        std::snprintf(names + 32 * q, 32, "%s", keys[q].c_str());
        launches[q] = cnt[q];
        total_ms[q] = tot[q];
    }
    *n_out = n;
    return CMM_OK;
}

int cmm_make_hashes(uint64_t seed, int32_t d, uint64_t *params) {
    g_err.clear();
    if (!params) return fail(CMM_ERR_ARG, "params is NULL");
    if (d < 1 || d > CMM_MAX_D) return fail(CMM_ERR_RANGE, "d = %d outside [1, %d]", d, CMM_MAX_D);
    uint64_t st = seed;
    for (int q = 0; q < 8 * d; ++q) params[q] = splitmix64(st);
    return CMM_OK;
}

size_t cmm_sketch_workspace_bytes(int64_t m, int64_t k, int64_t p, int32_t d, int32_t log2b,
                                  int32_t dtype, int32_t prec, int32_t transA) {
    if (m < 0 || k < 0 || p < 0 || d < 1 || d > CMM_MAX_D || log2b < 1 ||
        log2b > CMM_MAX_LOG2B || !valid_dtype(dtype))
        return 0;
    SketchPlan pl;
    if (!plan_sketch(m, k, p, d, log2b, dtype, prec, transA, transA ? m : k, p, pl)) return 0;
    return pl.total;
}

int cmm_sketch(const void *A, int64_t lda, int32_t transA, const void *B, int64_t ldb,
               int32_t dtype, int64_t m, int64_t k, int64_t p, const cmm_hashes *hs,
               int32_t prec, double *R, void *ws, size_t ws_bytes, void *stream) {
    g_err.clear();
    int rc = check_hashes(hs);
    if (rc) return rc;
    rc = check_operands(A, lda, transA, B, ldb, dtype, m, k, p, prec);
    if (rc) return rc;
    rc = check_prec_sizes(prec, hs->log2b, m, p);
    if (rc) return rc;
    if (!R) return fail(CMM_ERR_ARG, "R is NULL");
    const size_t need = cmm_sketch_workspace_bytes(m, k, p, hs->d, hs->log2b, dtype, prec, transA);
    rc = check_ws(ws, ws_bytes, need);
    if (rc) return rc;
    return run_sketch(A, lda, transA, B, ldb, dtype, m, k, p, hs, prec, R, ws,
                      static_cast<cudaStream_t>(stream));
}

size_t cmm_extract_workspace_bytes(int64_t m, int64_t p, int32_t d) {
    if (m < 0 || p < 0 || d < 1 || d > CMM_MAX_D) return 0;
    return extract_ws_bytes(m, p, d);
}

int cmm_extract(const double *R, const cmm_hashes *hs, int64_t m, int64_t p, int32_t reduce,
                double *C, int64_t ldc, void *ws, size_t ws_bytes, void *stream) {
    g_err.clear();
    int rc = check_hashes(hs);
    if (rc) return rc;
    rc = check_sizes(m, 0, p);
    if (rc) return rc;
    if (reduce != CMM_MEDIAN && reduce != CMM_MEAN) return fail(CMM_ERR_ARG, "bad reduce %d", reduce);
    if (m > 0 && p > 0) {
        if (!R || !C) return fail(CMM_ERR_ARG, "R or C is NULL");
        if (ldc < p) return fail(CMM_ERR_ARG, "ldc = %lld < p", (long long)ldc);
    }
    rc = check_ws(ws, ws_bytes, extract_ws_bytes(m, p, hs->d));
    if (rc) return rc;
    return run_extract(R, hs, m, p, reduce, C, ldc, ws, static_cast<cudaStream_t>(stream));
}

int cmm_heavy_hitters(const double *R, const cmm_hashes *hs, int64_t m, int64_t p,
                      int32_t reduce, double tau, int32_t *I, int32_t *J, double *V,
                      int64_t capacity, int64_t *count, void *ws, size_t ws_bytes,
                      void *stream) {
    g_err.clear();
    int rc = check_hashes(hs);
    if (rc) return rc;
    rc = check_sizes(m, 0, p);
    if (rc) return rc;
    if (reduce != CMM_MEDIAN && reduce != CMM_MEAN) return fail(CMM_ERR_ARG, "bad reduce %d", reduce);
    if (!count) return fail(CMM_ERR_ARG, "count is NULL");
    if (capacity < 0) return fail(CMM_ERR_ARG, "negative capacity");
    if (m > 0 && p > 0 && !R) return fail(CMM_ERR_ARG, "R is NULL");
    if (capacity > 0 && (!I || !J || !V)) return fail(CMM_ERR_ARG, "I, J or V is NULL");
    rc = check_ws(ws, ws_bytes, extract_ws_bytes(m, p, hs->d));
    if (rc) return rc;
    return run_hh_R(R, hs, m, p, reduce, tau, I, J, V, capacity, count, ws,
                    static_cast<cudaStream_t>(stream));
}

int cmm_threshold(const double *C, int64_t m, int64_t p, int64_t ldc, double tau, int32_t *I,
                  int32_t *J, double *V, int64_t capacity, int64_t *count, void *ws,
                  size_t ws_bytes, void *stream) {
    g_err.clear();
    int rc = check_sizes(m, 0, p);
    if (rc) return rc;
    if (!count) return fail(CMM_ERR_ARG, "count is NULL");
    if (capacity < 0) return fail(CMM_ERR_ARG, "negative capacity");
    if (m > 0 && p > 0 && (!C || ldc < p)) return fail(CMM_ERR_ARG, "C is NULL or ldc < p");
    if (capacity > 0 && (!I || !J || !V)) return fail(CMM_ERR_ARG, "I, J or V is NULL");
    rc = check_ws(ws, ws_bytes, extract_ws_bytes(m, p, 1));
    if (rc) return rc;
    return run_hh_dense(C, ldc, m, p, tau, I, J, V, capacity, count, ws,
                        static_cast<cudaStream_t>(stream));
}

size_t cmm_multiply_workspace_bytes(int64_t m, int64_t k, int64_t p, int32_t d, int32_t log2b,
                                    int32_t dtype, int32_t prec, int32_t transA) {
    const size_t sk = cmm_sketch_workspace_bytes(m, k, p, d, log2b, dtype, prec, transA);
    if (!sk) return 0;
    const size_t ex = extract_ws_bytes(m, p, d);
    return align_up((size_t)d * (size_t(1) << log2b) * sizeof(double)) + std::max(sk, ex);
}

int cmm_multiply(const void *A, int64_t lda, int32_t transA, const void *B, int64_t ldb,
                 int32_t dtype, int64_t m, int64_t k, int64_t p, const cmm_hashes *hs,
                 int32_t prec, int32_t reduce, double *C, int64_t ldc, double *R, void *ws,
                 size_t ws_bytes, void *stream) {
    g_err.clear();
    int rc = check_hashes(hs);
    if (rc) return rc;
    rc = check_operands(A, lda, transA, B, ldb, dtype, m, k, p, prec);
    if (rc) return rc;
    rc = check_prec_sizes(prec, hs->log2b, m, p);
    if (rc) return rc;
    if (reduce != CMM_MEDIAN && reduce != CMM_MEAN) return fail(CMM_ERR_ARG, "bad reduce %d", reduce);
    if (m > 0 && p > 0 && (!C || ldc < p)) return fail(CMM_ERR_ARG, "C is NULL or ldc < p");
    const size_t need = cmm_multiply_workspace_bytes(m, k, p, hs->d, hs->log2b, dtype, prec, transA);
    rc = check_ws(ws, ws_bytes, need);
    if (rc) return rc;
    char *base = static_cast<char *>(ws);
    const size_t rbytes = align_up((size_t)hs->d * (size_t(1) << hs->log2b) * sizeof(double));
    double *Rw = R ? R : reinterpret_cast<double *>(base);
    void *scratch = base + rbytes;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = run_sketch(A, lda, transA, B, ldb, dtype, m, k, p, hs, prec, Rw, scratch, s);
    if (rc) return rc;
    return run_extract(Rw, hs, m, p, reduce, C, ldc, scratch, s);
}

int cmm_multiply_threshold(const void *A, int64_t lda, int32_t transA, const void *B, int64_t ldb,
                           int32_t dtype, int64_t m, int64_t k, int64_t p, const cmm_hashes *hs,
                           int32_t prec, int32_t reduce, double *C, int64_t ldc, double *R,
                           double tau, int32_t *I, int32_t *J, double *V, int64_t capacity,
                           int64_t *count, void *ws, size_t ws_bytes, void *stream) {
    g_err.clear();
    if (!count) return fail(CMM_ERR_ARG, "count is NULL");
    *count = 0;
    if (capacity < 0) return fail(CMM_ERR_ARG, "negative capacity");
    if (capacity > 0 && (!I || !J || !V)) return fail(CMM_ERR_ARG, "I, J or V is NULL");
    int rc = check_hashes(hs);
    if (rc) return rc;
    rc = check_operands(A, lda, transA, B, ldb, dtype, m, k, p, prec);
    if (rc) return rc;
    rc = check_prec_sizes(prec, hs->log2b, m, p);
    if (rc) return rc;
    if (reduce != CMM_MEDIAN && reduce != CMM_MEAN) return fail(CMM_ERR_ARG, "bad reduce %d", reduce);
    if (m > 0 && p > 0 && (!C || ldc < p)) return fail(CMM_ERR_ARG, "C is NULL or ldc < p");
    const size_t need = cmm_multiply_workspace_bytes(m, k, p, hs->d, hs->log2b, dtype, prec, transA);
    rc = check_ws(ws, ws_bytes, need);
    if (rc) return rc;
    char *base = static_cast<char *>(ws);
    const size_t rbytes = align_up((size_t)hs->d * (size_t(1) << hs->log2b) * sizeof(double));
    double *Rw = R ? R : reinterpret_cast<double *>(base);
    void *scratch = base + rbytes;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = run_sketch(A, lda, transA, B, ldb, dtype, m, k, p, hs, prec, Rw, scratch, s);
    if (rc) return rc;
    if (m == 0 || p == 0) return CMM_OK;
    const HhRange hr = hh_range(tau);
    rc = run_extract(Rw, hs, m, p, reduce, C, ldc, scratch, s, 0, &hr);
    if (rc) return rc;
    return finish_hh(carve_extract(scratch, m, p, hs->d), true, C, ldc, m, p, hr, I, J, V,
                     capacity, count, s);
}

}  // extern "C"
