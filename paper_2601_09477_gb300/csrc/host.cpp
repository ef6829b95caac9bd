// host.cpp -- the C ABI of libcmm (include/cmm.h): argument checks, hash
// parameter generation, workspace planning and kernel launches.  No function
// here allocates device memory; every scratch byte comes from the caller's ws.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "cmm_internal.h"

using namespace cmm;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *where) {
    return fail(CMM_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int num_sms() {
    static int cached = 0;
    if (cached) return cached;
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0) {
        cached = n;
    } else {
        cudaGetLastError();   // no device here: plan for a GB300
        n = 152;
    }
    return n;
}

int check_hashes(const cmm_hashes *hs) {
    if (!hs || !hs->params) return fail(CMM_ERR_ARG, "hashes: null pointer");
    if (hs->d < 1 || hs->d > CMM_MAX_D)
        return fail(CMM_ERR_RANGE, "d = %d outside [1, %d]", hs->d, CMM_MAX_D);
    if (hs->log2b < 1 || hs->log2b > CMM_MAX_LOG2B)
        return fail(CMM_ERR_RANGE, "log2b = %d outside [1, %d]", hs->log2b, CMM_MAX_LOG2B);
    return CMM_OK;
}

void fill_params(const cmm_hashes *hs, HashParams &hp) {
    std::memset(&hp, 0, sizeof hp);
    for (int r = 0; r < hs->d; ++r) {
        const uint64_t *w = hs->params + 8 * r;
        hp.rep[r] = HashRep{w[0], w[1], w[2], w[3], w[4], w[5], w[6], w[7]};
    }
}

bool valid_dtype(int dt) { return dt == CMM_F64 || dt == CMM_F32 || dt == CMM_BF16; }
size_t dtype_size(int dt) { return dt == CMM_F64 ? 8 : dt == CMM_F32 ? 4 : 2; }

int check_sizes(int64_t m, int64_t k, int64_t p) {
    if (m < 0 || k < 0 || p < 0) return fail(CMM_ERR_ARG, "negative size");
    if (m >= (int64_t(1) << 31) || p >= (int64_t(1) << 31))
        return fail(CMM_ERR_RANGE, "m and p must be < 2^31 (hash keys are 32-bit row/column indices)");
    return CMM_OK;
}

// ---- sketch planning -------------------------------------------------------
bool plan_sketch(int64_t m, int64_t k, int64_t p, int d, int L, int dtype, int prec, int transA,
                 int64_t lda, int64_t ldb, SketchPlan &pl) {
    pl = SketchPlan{};
    pl.prec = prec;
    pl.L = L;
    const bool f64 = prec == CMM_PREC_F64;
    const int maxLlo = f64 ? kMaxLloF64 : kMaxLloF32;
    pl.Llo = std::min(L, maxLlo);
    pl.C = 1 << (L - pl.Llo);
    pl.threads = f64 ? sketch_threads_f64(pl.Llo) : sketch_threads_f32(pl.Llo);
    pl.smem = f64 ? sketch_smem_f64(pl.Llo) : sketch_smem_f32(pl.Llo);
    const int LE = std::min(pl.Llo, f64 ? 4 : 5);
    const int P = (1 << pl.Llo) >> LE;
    const int G = pl.threads / P;
    const int per_sm = pl.threads >= 512 ? 1 : 2;
    const int64_t slots = (int64_t)num_sms() * per_sm;
    const int64_t items = (int64_t)d * pl.C;

    // blocks of the inner index: at most 256 t per group (bounded FP32
    // accumulation), otherwise as few blocks as fill the GPU evenly
    const int64_t kk = std::max<int64_t>(k, 1);
    const int64_t nc_min = std::max<int64_t>(1, (kk + 256 * G - 1) / (256 * G));
    const int64_t nc_max = std::max<int64_t>(nc_min, (kk + G - 1) / G);
    int64_t best = nc_min;
    double best_eff = -1.0;
    for (int64_t nc = nc_min; nc <= std::min(nc_max, nc_min + 8 * slots); ++nc) {
        const int64_t total = items * nc;
        const int64_t waves = (total + slots - 1) / slots;
        const double eff = (double)total / (double)(waves * slots);
        if (eff > best_eff + 0.005) {
            best_eff = eff;
            best = nc;
        }
    }
    pl.chunk = (kk + best - 1) / best;
    pl.nchunks = (int)((kk + pl.chunk - 1) / pl.chunk);

    const size_t tb = f64 ? 8 : 4;
    const int tb_dtype = f64 ? CMM_F64 : CMM_F32;
    pl.prep_A = !(transA && dtype == tb_dtype);
    pl.prep_B = dtype != tb_dtype;
    pl.ldat = pl.prep_A ? m : lda;
    pl.ldbp = pl.prep_B ? p : ldb;
    const int64_t b = int64_t(1) << L;
    size_t off = 0;
    pl.off_At = off;
    if (pl.prep_A) off += align_up((size_t)k * m * tb);
    pl.off_Bp = off;
    if (pl.prep_B) off += align_up((size_t)k * p * tb);
    pl.off_partial = off;
    off += align_up((size_t)pl.nchunks * d * b * sizeof(double));
    pl.off_Z = off;
    off += align_up((size_t)d * b * sizeof(double));
    pl.total = off;
    return true;
}

int check_ws(void *ws, size_t ws_bytes, size_t need) {
    if (need == 0) return CMM_OK;
    if (!ws) return fail(CMM_ERR_WORKSPACE, "workspace is NULL but %zu bytes are needed", need);
    if (reinterpret_cast<uintptr_t>(ws) % kAlign)
        return fail(CMM_ERR_WORKSPACE, "workspace must be %zu-byte aligned", kAlign);
    if (ws_bytes < need)
        return fail(CMM_ERR_WORKSPACE, "workspace has %zu bytes, %zu needed", ws_bytes, need);
    return CMM_OK;
}

int check_operands(const void *A, int64_t lda, int transA, const void *B, int64_t ldb, int dtype,
                   int64_t m, int64_t k, int64_t p, int prec) {
    int rc = check_sizes(m, k, p);
    if (rc) return rc;
    if (!valid_dtype(dtype)) return fail(CMM_ERR_ARG, "bad dtype %d", dtype);
    if (prec != CMM_PREC_F64 && prec != CMM_PREC_F32 && prec != CMM_PREC_BF16TC)
        return fail(CMM_ERR_ARG, "bad precision %d", prec);
    if (transA != 0 && transA != 1) return fail(CMM_ERR_ARG, "transA must be 0 or 1");
    if (m > 0 && k > 0 && !A) return fail(CMM_ERR_ARG, "A is NULL");
    if (k > 0 && p > 0 && !B) return fail(CMM_ERR_ARG, "B is NULL");
    if (k > 0 && m > 0 && lda < (transA ? m : k))
        return fail(CMM_ERR_ARG, "lda = %lld too small", (long long)lda);
    if (k > 0 && p > 0 && ldb < p) return fail(CMM_ERR_ARG, "ldb = %lld too small", (long long)ldb);
    return CMM_OK;
}

size_t extract_ws_bytes(int64_t m, int64_t p, int d) {
    return align_up((size_t)d * m * 4) + align_up((size_t)d * p * 4) +
           align_up((size_t)(2 * m + 1) * sizeof(int64_t));
}

struct ExtractWs {
    uint32_t *H1, *H2;
    int64_t *counts;
};

ExtractWs carve_extract(void *ws, int64_t m, int64_t p, int d) {
    char *base = static_cast<char *>(ws);
    ExtractWs e;
    e.H1 = reinterpret_cast<uint32_t *>(base);
    base += align_up((size_t)d * m * 4);
    e.H2 = reinterpret_cast<uint32_t *>(base);
    base += align_up((size_t)d * p * 4);
    e.counts = reinterpret_cast<int64_t *>(base);
    return e;
}

int run_sketch(const void *A, int64_t lda, int transA, const void *B, int64_t ldb, int dtype,
               int64_t m, int64_t k, int64_t p, const cmm_hashes *hs, int prec, double *R,
               void *ws, cudaStream_t s) {
    SketchPlan pl;
    plan_sketch(m, k, p, hs->d, hs->log2b, dtype, prec, transA, lda, ldb, pl);
    HashParams hp;
    fill_params(hs, hp);
    char *base = static_cast<char *>(ws);
    const void *At = A, *Bp = B;
    cudaError_t e;
    if (pl.prep_A && m > 0 && k > 0) {
        e = launch_prep_A(A, lda, transA, dtype, prec, m, k, base + pl.off_At, pl.ldat, s);
        if (e != cudaSuccess) return cuda_fail(e, "prep A");
        At = base + pl.off_At;
    }
    if (pl.prep_B && p > 0 && k > 0) {
        e = launch_prep_B(B, ldb, dtype, prec, k, p, base + pl.off_Bp, pl.ldbp, s);
        if (e != cudaSuccess) return cuda_fail(e, "prep B");
        Bp = base + pl.off_Bp;
    }
    double *partial = reinterpret_cast<double *>(base + pl.off_partial);
    double *Z = reinterpret_cast<double *>(base + pl.off_Z);
    if (prec == CMM_PREC_F64)
        e = launch_sketch_f64(pl, (const double *)At, (const double *)Bp, m, k, p, hs->d, hp,
                              partial, s);
    else
        e = launch_sketch_f32(pl, (const float *)At, (const float *)Bp, m, k, p, hs->d, hp,
                              partial, s);
    if (e != cudaSuccess) return cuda_fail(e, "sketch kernel");
    e = launch_finish(partial, pl.nchunks, hs->d, hs->log2b, Z, R, s);
    if (e != cudaSuccess) return cuda_fail(e, "finish kernels");
    return CMM_OK;
}

int run_extract(const double *R, const cmm_hashes *hs, int64_t m, int64_t p, int reduce,
                double *C, int64_t ldc, void *ws, cudaStream_t s) {
    if (m == 0 || p == 0) return CMM_OK;
    HashParams hp;
    fill_params(hs, hp);
    ExtractWs ew = carve_extract(ws, m, p, hs->d);
    cudaError_t e = launch_hash_tables(hp, hs->d, hs->log2b, m, p, ew.H1, ew.H2, s);
    if (e != cudaSuccess) return cuda_fail(e, "hash tables");
    e = launch_extract(R, ew.H1, ew.H2, hs->d, hs->log2b, m, p, reduce, C, ldc, s);
    if (e != cudaSuccess) return cuda_fail(e, "extract kernel");
    return CMM_OK;
}

int run_hh(const double *R, const cmm_hashes *hs, const double *C, int64_t ldc, int64_t m,
           int64_t p, int d, int L, int reduce, double tau, int32_t *I, int32_t *J, double *V,
           int64_t capacity, int64_t *count, void *ws, cudaStream_t s) {
    *count = 0;
    if (m == 0 || p == 0) return CMM_OK;
    ExtractWs ew = carve_extract(ws, m, p, d);
    cudaError_t e;
    if (!C) {
        HashParams hp;
        fill_params(hs, hp);
        e = launch_hash_tables(hp, d, L, m, p, ew.H1, ew.H2, s);
        if (e != cudaSuccess) return cuda_fail(e, "hash tables");
    }
    e = launch_hh_count(R, ew.H1, ew.H2, C, ldc, d, L, m, p, reduce, tau, 1, m, ew.counts, s);
    if (e != cudaSuccess) return cuda_fail(e, "heavy-hitter count");
    e = launch_hh_scan(ew.counts, m, s);
    if (e != cudaSuccess) return cuda_fail(e, "heavy-hitter scan");
    int64_t total = 0;
    e = cudaMemcpyAsync(&total, ew.counts + 2 * m, sizeof total, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "heavy-hitter count copy");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "heavy-hitter count sync");
    *count = total;
    if (total > 0 && capacity > 0) {
        e = launch_hh_write(R, ew.H1, ew.H2, C, ldc, d, L, m, p, reduce, tau, 1, m,
                            ew.counts + m, I, J, V, capacity, s);
        if (e != cudaSuccess) return cuda_fail(e, "heavy-hitter write");
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "heavy-hitter write sync");
    }
    if (total > capacity)
        return fail(CMM_ERR_CAPACITY, "%lld heavy hitters, capacity %lld", (long long)total,
                    (long long)capacity);
    return CMM_OK;
}

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
    plan_sketch(m, k, p, d, log2b, dtype, prec, transA, transA ? m : k, p, pl);
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
    if (prec == CMM_PREC_BF16TC)
        return fail(CMM_ERR_ARG, "precision BF16TC is not available in this build");
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
    return run_hh(R, hs, nullptr, 0, m, p, hs->d, hs->log2b, reduce, tau, I, J, V, capacity, count,
                  ws, static_cast<cudaStream_t>(stream));
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
    return run_hh(nullptr, nullptr, C, ldc, m, p, 1, 1, CMM_MEDIAN, tau, I, J, V, capacity, count,
                  ws, static_cast<cudaStream_t>(stream));
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
    if (prec == CMM_PREC_BF16TC)
        return fail(CMM_ERR_ARG, "precision BF16TC is not available in this build");
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

int cmm_mean_pairs(const double *R, const cmm_hashes *hs, int64_t P, const int32_t *I,
                   const int32_t *J, double *out, void *stream) {
    g_err.clear();
    int rc = check_hashes(hs);
    if (rc) return rc;
    if (P < 0) return fail(CMM_ERR_ARG, "negative pair count");
    if (P == 0) return CMM_OK;
    if (!R || !I || !J || !out) return fail(CMM_ERR_ARG, "null pointer");
    HashParams hp;
    fill_params(hs, hp);
    cudaError_t e = launch_mean_pairs(R, hp, hs->d, hs->log2b, P, I, J, out,
                                      static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "mean pairs");
    return CMM_OK;
}

}  // extern "C"
