// api_adjoint.cpp -- the differentiable mean estimator: cmm_mean_pairs
// (forward at a list of pairs) and cmm_backward (its adjoint).
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

// ---- adjoint planning --------------------------------------------------------
constexpr size_t kMaxDynSmem = 227 * 1024;

bool plan_adjoint(int64_t m, int64_t k, int64_t p, int d, int L, int dtype, int prec, int transA,
                  int64_t lda, int64_t ldb, AdjointPlan &pl) {
    pl = AdjointPlan{};
    pl.prec = prec;
    pl.L = L;
    const bool f64 = prec == CMM_PREC_F64;
    pl.Llo = std::min(L, f64 ? kMaxLloF64 : kMaxLloF32);
    pl.C = 1 << (L - pl.Llo);
    pl.threads = adjoint_threads(prec, pl.Llo);
    const int LE = std::min(pl.Llo, f64 ? 4 : 5);
    const int N = 1 << pl.Llo;
    const int P = N >> LE;
    const int G = pl.threads / P;
    const size_t es = f64 ? 8 : 4;
    const int pad = (!f64 && LE == 5) ? 4 : 1;   // shared-memory pad words per row
    pl.smem = (size_t)G * ((size_t)N + (size_t)pad * (N >> LE) + m + p) * es;
    int64_t slots = num_sms();
    int Gt = G;
    if (!f64 && pl.Llo == adjoint_tm_llo() && adjoint_tm_smem(m, p) <= kMaxDynSmem) {
        // the tensor-memory kernel: 128 threads, two CTAs per SM when their
        // shared memory allows
        pl.tm = true;
        pl.threads = adjoint_tm_threads();
        pl.smem = adjoint_tm_smem(m, p);
        Gt = 1;
        if (2 * pl.smem <= kMaxDynSmem) slots *= 2;
    }
    if (pl.smem > kMaxDynSmem) return false;
    const int64_t kk = std::max<int64_t>(k, 1);
    const int64_t nc_max = std::max<int64_t>(1, (kk + Gt - 1) / Gt);
    int64_t best = 1;
    double best_eff = -1.0;
    for (int64_t nc = 1; nc <= std::min<int64_t>(nc_max, 8 * slots); ++nc) {
        const int64_t total = (int64_t)pl.C * nc;
        const int64_t waves = (total + slots - 1) / slots;
        const double eff = (double)total / (double)(waves * slots);
        if (eff > best_eff + 0.005) {
            best_eff = eff;
            best = nc;
        }
    }
    pl.chunk = (kk + best - 1) / best;
    pl.nchunks = (int)((kk + pl.chunk - 1) / pl.chunk);
    const int tb_dtype = f64 ? CMM_F64 : CMM_F32;
    pl.prep_A = !(transA && dtype == tb_dtype);
    pl.prep_B = dtype != tb_dtype;
    pl.ldat = pl.prep_A ? m : lda;
    pl.ldbp = pl.prep_B ? p : ldb;
    const size_t bb = (size_t)d * ((size_t)1 << L) * sizeof(double);
    size_t off = 0;
    pl.off_At = off;
    if (pl.prep_A) off += align_up((size_t)k * m * es);
    pl.off_Bp = off;
    if (pl.prep_B) off += align_up((size_t)k * p * es);
    pl.off_G = off;
    off += align_up(bb);
    pl.off_Gs = off;
    off += align_up(bb);
    pl.off_Z = off;
    off += align_up(bb);
    pl.off_dAt = off;
    off += align_up((size_t)k * m * es);
    pl.off_dBt = off;
    off += align_up((size_t)k * p * es);
    pl.off_colmax = off;
    if (!f64) off += align_up((size_t)2 * k * sizeof(float));
    if (pl.tm) {
        pl.off_tabA = off;
        off += align_up((size_t)d * pl.C * m * sizeof(tab_t));
        pl.off_tabB = off;
        off += align_up((size_t)d * pl.C * p * sizeof(tab_t));
        pl.off_Gs32 = off;
        off += align_up((size_t)d * ((size_t)1 << L) * sizeof(float));
    }
    pl.total = off;
    return true;
}

}  // namespace

extern "C" {

size_t cmm_backward_workspace_bytes(int64_t m, int64_t k, int64_t p, int32_t d, int32_t log2b,
                                    int32_t dtype, int32_t prec, int32_t transA) {
    if (m < 0 || k < 0 || p < 0 || d < 1 || d > CMM_MAX_D || log2b < 1 ||
        log2b > CMM_MAX_LOG2B || (dtype != CMM_F64 && dtype != CMM_F32) ||
        (prec != CMM_PREC_F64 && prec != CMM_PREC_F32))
        return 0;
    AdjointPlan pl;
    if (!plan_adjoint(m, k, p, d, log2b, dtype, prec, transA, transA ? m : k, p, pl)) return 0;
    return pl.total;
}

int cmm_backward(const void *A, int64_t lda, int32_t transA, const void *B, int64_t ldb,
                 int32_t dtype, int64_t m, int64_t k, int64_t p, const cmm_hashes *hs,
                 int32_t prec, int64_t P, const int32_t *I, const int32_t *J, const double *W,
                 void *dA, int64_t ldda, void *dB, int64_t lddb, void *ws, size_t ws_bytes,
                 void *stream) {
    g_err.clear();
    int rc = check_hashes(hs);
    if (rc) return rc;
    rc = check_operands(A, lda, transA, B, ldb, dtype, m, k, p, prec);
    if (rc) return rc;
    if (dtype == CMM_BF16) return fail(CMM_ERR_ARG, "cmm_backward takes FP32 or FP64 operands");
    if (prec != CMM_PREC_F64 && prec != CMM_PREC_F32)
        return fail(CMM_ERR_ARG, "cmm_backward supports the FP64 and FP32 precisions");
    if (P < 0) return fail(CMM_ERR_ARG, "negative pair count");
    if (P > 0 && (!I || !J || !W)) return fail(CMM_ERR_ARG, "I, J or W is NULL");
    if (m > 0 && k > 0 && (!dA || ldda < (transA ? m : k))) return fail(CMM_ERR_ARG, "dA is NULL or ldda too small");
    if (k > 0 && p > 0 && (!dB || lddb < p)) return fail(CMM_ERR_ARG, "dB is NULL or lddb too small");
    AdjointPlan pl;
    if (!plan_adjoint(m, k, p, hs->d, hs->log2b, dtype, prec, transA, lda, ldb, pl))
        return fail(CMM_ERR_RANGE, "cmm_backward: m + p too large for the on-chip gradient rows");
    rc = check_ws(ws, ws_bytes, pl.total);
    if (rc) return rc;
    if (m == 0 || k == 0 || p == 0) {
        // empty gradient: nothing to compute (dA / dB have no entries or are zero)
        cudaStream_t s0 = static_cast<cudaStream_t>(stream);
        const size_t es = dtype == CMM_F64 ? 8 : 4;
        cudaError_t e = cudaSuccess;
        if (m > 0 && k > 0)
            e = cudaMemset2DAsync(dA, ldda * es, 0, (transA ? m : k) * es, transA ? k : m, s0);
        if (e == cudaSuccess && k > 0 && p > 0)
            e = cudaMemset2DAsync(dB, lddb * es, 0, p * es, k, s0);
        return e == cudaSuccess ? CMM_OK : cuda_fail(e, "zero gradients");
    }
    HashParams hp;
    fill_params(hs, hp);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(ws);
    const void *At = A, *Bp = B;
    cudaError_t e;
    if (pl.prep_A) {
        Span sp("prep_A", s);
        e = launch_prep_A(A, lda, transA, dtype, prec, m, k, base + pl.off_At, pl.ldat, s);
        if (e != cudaSuccess) return cuda_fail(e, "prep A");
        At = base + pl.off_At;
    }
    if (pl.prep_B) {
        Span sp("prep_B", s);
        e = launch_prep_B(B, ldb, dtype, prec, k, p, base + pl.off_Bp, pl.ldbp, s);
        if (e != cudaSuccess) return cuda_fail(e, "prep B");
        Bp = base + pl.off_Bp;
    }
    double *G = reinterpret_cast<double *>(base + pl.off_G);
    double *Gs = reinterpret_cast<double *>(base + pl.off_Gs);
    double *Z = reinterpret_cast<double *>(base + pl.off_Z);
    {
        Span sp("adj_g", s);
        e = launch_adj_g(hp, hs->d, hs->log2b, P, I, J, W, G, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "adjoint weights");
    {
        Span sp("finish", s, 2);
        e = launch_finish(G, 1, hs->d, hs->log2b, Z, Gs, s);   // Gs = (1/b) H G
    }
    if (e != cudaSuccess) return cuda_fail(e, "adjoint weight transform");
    void *dAt = base + pl.off_dAt, *dBt = base + pl.off_dBt;
    float *colmax = reinterpret_cast<float *>(base + pl.off_colmax);
    if (prec == CMM_PREC_F32) {
        Span sp("colmax", s, 2);
        e = launch_rowmax((const float *)At, pl.ldat, k, m, colmax, s);
        if (e == cudaSuccess) e = launch_rowmax((const float *)Bp, pl.ldbp, k, p, colmax + k, s);
        if (e != cudaSuccess) return cuda_fail(e, "column maxima");
    }
    {
        Span sp(prec == CMM_PREC_F64 ? "adjoint_f64" : "adjoint_f32", s, pl.tm ? 3 : 1);
        if (pl.tm)
            e = launch_adjoint_tm(pl, (const float *)At, (const float *)Bp, m, k, p, hs->d, hp,
                                  Gs, reinterpret_cast<float *>(base + pl.off_Gs32),
                                  reinterpret_cast<tab_t *>(base + pl.off_tabA),
                                  reinterpret_cast<tab_t *>(base + pl.off_tabB), colmax,
                                  (float *)dAt, (float *)dBt, s);
        else
            e = launch_adjoint(pl, At, Bp, m, k, p, hs->d, hp, Gs, colmax, dAt, dBt, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "adjoint kernel");
    {
        Span sp("grad_out", s, 2);
        const int f64 = prec == CMM_PREC_F64;
        // dAt is k x m: dA has A's layout (A^T stored when transA)
        e = launch_convert_out(dAt, f64, k, m, transA ? 0 : 1, dA, dtype, ldda, s);
        if (e == cudaSuccess) e = launch_convert_out(dBt, f64, k, p, 0, dB, dtype, lddb, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "gradient output");
    return CMM_OK;
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
    cudaError_t e;
    {
        Span sp("mean_pairs", static_cast<cudaStream_t>(stream));
        e = launch_mean_pairs(R, hp, hs->d, hs->log2b, P, I, J, out,
                              static_cast<cudaStream_t>(stream));
    }
    if (e != cudaSuccess) return cuda_fail(e, "mean pairs");
    return CMM_OK;
}

}  // extern "C"
