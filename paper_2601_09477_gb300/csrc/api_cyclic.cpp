// api_cyclic.cpp -- Pagh's original cyclic form (Sec. 3.1) through the FFT:
// planning, Compress, Decompress and multiply.
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

// ---- the cyclic (FFT) form of Sec. 3.1 --------------------------------------
bool plan_cyclic(int64_t m, int64_t k, int64_t p, int d, int L, int dtype, int transA,
                 int64_t lda, int64_t ldb, SketchPlan &pl) {
    pl = SketchPlan{};
    if (L < sketch_fft_llo()) return false;
    pl.prec = CMM_PREC_F32;
    pl.L = L;
    pl.Llo = sketch_fft_llo();
    pl.C = 1 << (L - pl.Llo);
    pl.nclass = pl.C / 2 + 1 < pl.C ? pl.C / 2 + 1 : pl.C;   // classes 0 .. C/2
    pl.threads = sketch_fft_threads();
    pl.smem = sketch_fft_smem();
    pl.nparts = 1;
    const int64_t slots = (int64_t)num_sms() * 2;
    const int64_t items = (int64_t)d * pl.nclass;
    const int64_t kk = std::max<int64_t>(k, 1);
    const int64_t nc_min = std::max<int64_t>(1, (kk + 255) / 256);
    int64_t best = nc_min;
    double best_cost = 1e300;
    for (int64_t nc = nc_min; nc <= std::min(kk, nc_min + 8 * slots); ++nc) {
        const int64_t waves = (items * nc + slots - 1) / slots;
        const double cost = (double)waves * (double)((kk + nc - 1) / nc + 2);
        if (cost < best_cost * 0.995) {
            best_cost = cost;
            best = nc;
        }
    }
    pl.chunk = (kk + best - 1) / best;
    pl.nchunks = (int)((kk + pl.chunk - 1) / pl.chunk);
    pl.kb[0] = 0;
    pl.kb[1] = k;
    pl.pchunk[0] = pl.chunk;
    pl.pnch[0] = pl.nchunks;
    pl.prep_A = !(transA && dtype == CMM_F32);
    pl.prep_B = dtype != CMM_F32;
    pl.ldat = pl.prep_A ? m : lda;
    pl.ldbp = pl.prep_B ? p : ldb;
    const int64_t N = int64_t(1) << pl.Llo;
    size_t off = 0;
    pl.off_At = off;
    if (pl.prep_A) off += align_up((size_t)k * m * 4);
    pl.off_Bp = off;
    if (pl.prep_B) off += align_up((size_t)k * p * 4);
    pl.off_partial = off;   // complex FP64 partials [block][r][class][N]
    off += align_up((size_t)pl.nchunks * d * pl.nclass * N * 16);
    pl.off_Z = off;         // G: per-class inverse transforms [r][C][N], complex FP64
    off += align_up((size_t)d * pl.C * N * 16);
    pl.off_tab = off;
    off += align_up((size_t)d * pl.nclass * (m + p) * sizeof(uint32_t));
    pl.off_colmax = off;
    off += align_up((size_t)2 * k * sizeof(float));
    pl.total = off;
    return true;
}

int run_sketch_cyclic(const void *A, int64_t lda, int transA, const void *B, int64_t ldb,
                      int dtype, int64_t m, int64_t k, int64_t p, const cmm_hashes *hs, double *R,
                      void *ws, cudaStream_t s) {
    SketchPlan pl;
    plan_cyclic(m, k, p, hs->d, hs->log2b, dtype, transA, lda, ldb, pl);
    HashParams hp;
    fill_params(hs, hp);
    char *base = static_cast<char *>(ws);
    const void *At = A, *Bp = B;
    cudaError_t e;
    if (pl.prep_A && m > 0 && k > 0) {
        Span sp("prep_A", s);
        e = launch_prep_A(A, lda, transA, dtype, CMM_PREC_F32, m, k, base + pl.off_At, pl.ldat, s);
        if (e != cudaSuccess) return cuda_fail(e, "prep A");
        At = base + pl.off_At;
    }
    if (pl.prep_B && p > 0 && k > 0) {
        Span sp("prep_B", s);
        e = launch_prep_B(B, ldb, dtype, CMM_PREC_F32, k, p, base + pl.off_Bp, pl.ldbp, s);
        if (e != cudaSuccess) return cuda_fail(e, "prep B");
        Bp = base + pl.off_Bp;
    }
    float *colmax = reinterpret_cast<float *>(base + pl.off_colmax);
    {
        Span sp("colmax", s, 2);
        e = launch_rowmax((const float *)At, pl.ldat, k, m, colmax, s);
        if (e == cudaSuccess) e = launch_rowmax((const float *)Bp, pl.ldbp, k, p, colmax + k, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "column maxima");
    uint32_t *tabA = reinterpret_cast<uint32_t *>(base + pl.off_tab);
    uint32_t *tabB = tabA + (size_t)hs->d * pl.nclass * m;
    double *partial = reinterpret_cast<double *>(base + pl.off_partial);
    {
        Span sp("sketch_cyclic", s, 2);   // tables, then the sketch kernel
        e = launch_sketch_fft(pl, (const float *)At, (const float *)Bp, m, k, p, hs->d, hp, tabA,
                              tabB, colmax, partial, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "cyclic sketch kernel");
    {
        Span sp("finish_cyclic", s, 2);
        e = launch_finish_fft(partial, pl.nchunks, hs->d, hs->log2b, pl.C, pl.nclass,
                              reinterpret_cast<double *>(base + pl.off_Z), R, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "cyclic finish kernels");
    return CMM_OK;
}

}  // namespace

extern "C" {

size_t cmm_sketch_cyclic_workspace_bytes(int64_t m, int64_t k, int64_t p, int32_t d,
                                         int32_t log2b, int32_t dtype, int32_t prec,
                                         int32_t transA) {
    if (m < 0 || k < 0 || p < 0 || d < 1 || d > CMM_MAX_D || log2b < 1 ||
        log2b > CMM_MAX_LOG2B || !valid_dtype(dtype) || prec != CMM_PREC_F32)
        return 0;
    SketchPlan pl;
    if (!plan_cyclic(m, k, p, d, log2b, dtype, transA, transA ? m : k, p, pl)) return 0;
    return pl.total;
}

int cmm_sketch_cyclic(const void *A, int64_t lda, int32_t transA, const void *B, int64_t ldb,
                      int32_t dtype, int64_t m, int64_t k, int64_t p, const cmm_hashes *hs,
                      int32_t prec, double *R, void *ws, size_t ws_bytes, void *stream) {
    g_err.clear();
    int rc = check_hashes(hs);
    if (rc) return rc;
    rc = check_operands(A, lda, transA, B, ldb, dtype, m, k, p, prec);
    if (rc) return rc;
    if (prec != CMM_PREC_F32) return fail(CMM_ERR_ARG, "the cyclic form runs FP32 butterflies only");
    if (hs->log2b < sketch_fft_llo())
        return fail(CMM_ERR_RANGE, "the cyclic form needs log2b >= %d", sketch_fft_llo());
    if (!R) return fail(CMM_ERR_ARG, "R is NULL");
    rc = check_ws(ws, ws_bytes,
                  cmm_sketch_cyclic_workspace_bytes(m, k, p, hs->d, hs->log2b, dtype, prec, transA));
    if (rc) return rc;
    return run_sketch_cyclic(A, lda, transA, B, ldb, dtype, m, k, p, hs, R, ws,
                             static_cast<cudaStream_t>(stream));
}

int cmm_extract_cyclic(const double *R, const cmm_hashes *hs, int64_t m, int64_t p,
                       int32_t reduce, double *C, int64_t ldc, void *ws, size_t ws_bytes,
                       void *stream) {
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
    return run_extract(R, hs, m, p, reduce, C, ldc, ws, static_cast<cudaStream_t>(stream), 1);
}

size_t cmm_multiply_cyclic_workspace_bytes(int64_t m, int64_t k, int64_t p, int32_t d,
                                           int32_t log2b, int32_t dtype, int32_t prec,
                                           int32_t transA) {
    const size_t sk = cmm_sketch_cyclic_workspace_bytes(m, k, p, d, log2b, dtype, prec, transA);
    if (!sk) return 0;
    const size_t ex = extract_ws_bytes(m, p, d);
    return align_up((size_t)d * (size_t(1) << log2b) * sizeof(double)) + std::max(sk, ex);
}

int cmm_multiply_cyclic(const void *A, int64_t lda, int32_t transA, const void *B,
                        int64_t ldb, int32_t dtype, int64_t m, int64_t k, int64_t p,
                        const cmm_hashes *hs, int32_t prec, int32_t reduce, double *C,
                        int64_t ldc, double *R, void *ws, size_t ws_bytes, void *stream) {
    g_err.clear();
    int rc = check_hashes(hs);
    if (rc) return rc;
    rc = check_operands(A, lda, transA, B, ldb, dtype, m, k, p, prec);
    if (rc) return rc;
    if (prec != CMM_PREC_F32) return fail(CMM_ERR_ARG, "the cyclic form runs FP32 butterflies only");
    if (hs->log2b < sketch_fft_llo())
        return fail(CMM_ERR_RANGE, "the cyclic form needs log2b >= %d", sketch_fft_llo());
    if (reduce != CMM_MEDIAN && reduce != CMM_MEAN) return fail(CMM_ERR_ARG, "bad reduce %d", reduce);
    if (m > 0 && p > 0 && (!C || ldc < p)) return fail(CMM_ERR_ARG, "C is NULL or ldc < p");
    rc = check_ws(ws, ws_bytes,
                  cmm_multiply_cyclic_workspace_bytes(m, k, p, hs->d, hs->log2b, dtype, prec,
                                                      transA));
    if (rc) return rc;
    char *base = static_cast<char *>(ws);
    const size_t rbytes = align_up((size_t)hs->d * (size_t(1) << hs->log2b) * sizeof(double));
    double *Rw = R ? R : reinterpret_cast<double *>(base);
    void *scratch = base + rbytes;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = run_sketch_cyclic(A, lda, transA, B, ldb, dtype, m, k, p, hs, Rw, scratch, s);
    if (rc) return rc;
    return run_extract(Rw, hs, m, p, reduce, C, ldc, scratch, s, 1);
}

}  // extern "C"
