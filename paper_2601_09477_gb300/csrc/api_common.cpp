// api_common.cpp -- the helpers of api_common.h: error text, launch tracing,
// argument checks, sketch planning and the Compress / Decompress /
// heavy-hitter drivers.  No function here allocates device memory; every
// scratch byte comes from the caller's workspace.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "api_common.h"

namespace cmm {
namespace api {

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

// ---- launch tracing: CUDA events around every kernel launch while enabled ----
std::mutex g_tr_mu;
bool g_tr_on = false;
std::vector<TraceRec> g_tr;
std::vector<cudaEvent_t> g_ev_pool;

cudaEvent_t tr_event() {
    cudaEvent_t e = nullptr;
    if (!g_ev_pool.empty()) {
        e = g_ev_pool.back();
        g_ev_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        e = nullptr;
    }
    return e;
}

// SM count of the current device, cached per device index (the plans size
// grids by it, so a process with GPUs of different sizes plans each for its own)
int num_sms() {
    constexpr int kDevs = 64;
    static std::atomic<int> cached[kDevs];
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();   // no device here: plan for a GB300
        return 152;
    }
    if (dev >= 0 && dev < kDevs) {
        const int c = cached[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        return 152;
    }
    if (dev >= 0 && dev < kDevs) cached[dev].store(n, std::memory_order_relaxed);
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

// The FP32 sketch of 2^14-point slices runs the TMEM kernel unless the
// environment sets CMM_SKETCH_KERNEL=regs (the register-only kernel; both are
// kept and tested against the oracle).
bool use_tmem_kernel() {
    static int cached = -1;
    if (cached < 0) {
        const char *v = std::getenv("CMM_SKETCH_KERNEL");
        cached = (v && std::strcmp(v, "regs") == 0) ? 0 : 1;
    }
    return cached == 1;
}

// ---- sketch planning -------------------------------------------------------
bool plan_sketch(int64_t m, int64_t k, int64_t p, int d, int L, int dtype, int prec, int transA,
                 int64_t lda, int64_t ldb, SketchPlan &pl, int nparts, double ratio) {
    pl = SketchPlan{};
    pl.prec = prec;
    pl.L = L;
    const bool fx = prec == CMM_PREC_FX64;   // exact fixed point: FP64 operands, int64 copies
    const bool tern = prec == CMM_PREC_TERNARY;   // packed pairs of rows, 2^14 slices
    const bool f64 = prec == CMM_PREC_F64 || fx;
    const bool bf16 = prec_tc(prec);
    if (bf16 && L < sketch_bf16_llo()) return false;
    if (tern && L < kMaxLloF32) return false;
    const int maxLlo = bf16 ? sketch_bf16_llo()
                            : fx ? kMaxLloFx64 : (f64 ? kMaxLloF64 : kMaxLloF32);
    pl.Llo = std::min(L, maxLlo);
    pl.C = 1 << (L - pl.Llo);
    pl.tmem = sketch_tm_supported(prec, pl.Llo) && use_tmem_kernel();
    pl.threads = bf16 ? sketch_bf16_threads()
                 : fx ? sketch_fx64_threads(pl.Llo)
                 : tern ? sketch_i16_threads()
                 : pl.tmem ? sketch_tm_threads()
                           : (f64 ? sketch_threads_f64(pl.Llo) : sketch_threads_f32(pl.Llo));
    pl.smem = bf16 ? sketch_bf16_smem()
              : fx ? sketch_fx64_smem(pl.Llo)
              : tern ? sketch_i16_smem()
              : pl.tmem ? sketch_tm_smem()
                        : (f64 ? sketch_smem_f64(pl.Llo) : sketch_smem_f32(pl.Llo));
    const int LE = bf16 ? pl.Llo : (pl.tmem || tern) ? 7 : std::min(pl.Llo, (f64 && !fx) ? 4 : 5);
    const int P = (1 << pl.Llo) >> LE;
    const int G = bf16 ? 1 : pl.threads / P;
    const int per_sm = bf16 ? 1 : (pl.tmem || pl.threads < 512) ? 2 : 1;
    const int64_t slots = (int64_t)num_sms() * per_sm;
    const int64_t items = (int64_t)d * pl.C;

    // blocks of the inner index, per part: at most 256 t per group (bounded
    // FP32 accumulation); otherwise the count that minimises the modelled
    // time waves * (t per group + a fixed per-CTA cost of ~2 t for the
    // partial write-out and set-up), preferring fewer blocks on ties
    nparts = std::max(1, std::min(nparts, kMaxParts));
    if (k < nparts || tern) nparts = 1;   // the ternary form plans in pairs of t, one part
    pl.nparts = nparts;
    pl.nchunks = 0;
    if (ratio > 0.0 && nparts > 1) {
        double w[kMaxParts + 1] = {0.0};
        for (int c = 0; c < nparts; ++c) w[c + 1] = w[c] + std::pow(ratio, c);
        pl.kb[0] = 0;
        for (int c = 1; c < nparts; ++c)
            pl.kb[c] = std::min<int64_t>(k - (nparts - c),
                                         std::max<int64_t>(pl.kb[c - 1] + 1,
                                                           (int64_t)(k * w[c] / w[nparts])));
        pl.kb[nparts] = k;
    } else {
        for (int c = 0; c <= nparts; ++c) pl.kb[c] = k * c / nparts;
    }
    for (int c = 0; c < nparts; ++c) {
        const int64_t kt = pl.kb[c + 1] - pl.kb[c];
        const int64_t kk = std::max<int64_t>(tern ? (kt + 1) / 2 : kt, 1);
        const int64_t nc_min = std::max<int64_t>(1, (kk + 256 * G - 1) / (256 * G));
        const int64_t nc_max = std::max<int64_t>(nc_min, (kk + G - 1) / G);
        int64_t best = nc_min;
        double best_cost = 1e300;
        for (int64_t nc = nc_min; nc <= std::min(nc_max, nc_min + 8 * slots); ++nc) {
            const int64_t waves = (items * nc + slots - 1) / slots;
            const int64_t per_group = ((kk + nc - 1) / nc + G - 1) / G;
            const double cost = (double)waves * (double)(per_group + 2);
            if (cost < best_cost * 0.995) {
                best_cost = cost;
                best = nc;
            }
        }
        pl.pchunk[c] = (kk + best - 1) / best;
        pl.pnch[c] = (int)((kk + pl.pchunk[c] - 1) / pl.pchunk[c]);
        pl.nchunks += pl.pnch[c];
    }
    pl.chunk = pl.pchunk[0];

    const size_t tb = f64 ? 8 : 4;
    const int tb_dtype = f64 ? CMM_F64 : CMM_F32;
    pl.prep_A = !(transA && (dtype == tb_dtype || (tern && dtype == CMM_F64)));
    pl.prep_B = tern ? dtype == CMM_BF16 : dtype != tb_dtype;   // packing reads FP64 and FP32
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
    pl.off_tab = off;
    off += align_up((size_t)d * pl.C * (m + p) * sizeof(tab_t));
    pl.off_colmax = off;
    if (!f64) off += align_up((size_t)2 * k * sizeof(float));
    pl.off_Aq = off;
    if (fx) off += align_up((size_t)k * m * sizeof(long long));
    pl.off_Bq = off;
    if (fx) off += align_up((size_t)k * p * sizeof(long long));
    pl.off_exp = off;
    if (fx) off += align_up((size_t)2 * k * sizeof(int));
    const int64_t pairs = (k + 1) / 2;
    pl.off_Ap2 = off;
    if (tern) off += align_up((size_t)pairs * m * sizeof(int));
    pl.off_Bp2 = off;
    if (tern) off += align_up((size_t)pairs * p * sizeof(int));
    pl.off_bad = off;
    if (tern) off += align_up(sizeof(int));
    pl.total = off;
    return true;
}

// size limits of the forms whose slices are fixed: the tensor-core forms and
// the ternary form transform whole slices (log2b at least one slice), and the
// ternary form's 16-bit halves hold sums of at most m (or p) entries
int check_prec_sizes(int prec, int log2b, int64_t m, int64_t p) {
    if (prec_tc(prec) && log2b < sketch_bf16_llo())
        return fail(CMM_ERR_RANGE, "the tensor-core precisions need log2b >= %d", sketch_bf16_llo());
    if (prec == CMM_PREC_TERNARY) {
        if (log2b < kMaxLloF32)
            return fail(CMM_ERR_RANGE, "the ternary form needs log2b >= %d", kMaxLloF32);
        if (m >= 32768 || p >= 32768)
            return fail(CMM_ERR_RANGE, "the ternary form needs m, p < 2^15 (16-bit halves)");
    }
    return CMM_OK;
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
    if (prec != CMM_PREC_F64 && prec != CMM_PREC_F32 && !prec_tc(prec) && prec != CMM_PREC_FX64 &&
        prec != CMM_PREC_TERNARY)
        return fail(CMM_ERR_ARG, "bad precision %d", prec);
    if (transA != 0 && transA != 1) return fail(CMM_ERR_ARG, "transA must be 0 or 1");
    if (m > 0 && k > 0 && !A) return fail(CMM_ERR_ARG, "A is NULL");
    if (k > 0 && p > 0 && !B) return fail(CMM_ERR_ARG, "B is NULL");
    if (k > 0 && m > 0 && lda < (transA ? m : k))
        return fail(CMM_ERR_ARG, "lda = %lld too small", (long long)lda);
    if (k > 0 && p > 0 && ldb < p) return fail(CMM_ERR_ARG, "ldb = %lld too small", (long long)ldb);
    return CMM_OK;
}

// candidates of the one-pass heavy-hitter list from R: one per 64 entries of
// the estimate, within [2^16, 2^24] (more hits fall back to a second pass)
int64_t hh_cand_capacity(int64_t m, int64_t p) {
    const double e = (double)m * (double)p / 64.0;
    return (int64_t)std::min(16777216.0, std::max(65536.0, e));
}

// extraction workspace: hash words of rows and columns, per-row counts and
// offsets (2m + 1), per-(row, tile) counts and candidate offsets of the
// heavy-hitter passes, the candidate counter and the candidates (i, j, value)
size_t extract_ws_bytes(int64_t m, int64_t p, int d) {
    const size_t mt = (size_t)m * hh_tiles(p);
    const size_t cc = (size_t)hh_cand_capacity(m, p);
    return align_up((size_t)d * m * 4) + align_up((size_t)d * p * 4) +
           align_up((size_t)(2 * m + 1) * sizeof(int64_t)) + align_up(mt * sizeof(int32_t)) +
           align_up(mt * sizeof(int64_t)) + align_up(sizeof(unsigned long long)) +
           2 * align_up(cc * sizeof(int32_t)) + align_up(cc * sizeof(double));
}

ExtractWs carve_extract(void *ws, int64_t m, int64_t p, int d) {
    char *base = static_cast<char *>(ws);
    ExtractWs e;
    e.nt = hh_tiles(p);
    e.ccap = hh_cand_capacity(m, p);
    const size_t mt = (size_t)m * e.nt;
    e.H1 = reinterpret_cast<uint32_t *>(base);
    base += align_up((size_t)d * m * 4);
    e.H2 = reinterpret_cast<uint32_t *>(base);
    base += align_up((size_t)d * p * 4);
    e.counts = reinterpret_cast<int64_t *>(base);
    base += align_up((size_t)(2 * m + 1) * sizeof(int64_t));
    e.tcounts = reinterpret_cast<int32_t *>(base);
    base += align_up(mt * sizeof(int32_t));
    e.tsrc = reinterpret_cast<int64_t *>(base);
    base += align_up(mt * sizeof(int64_t));
    e.ncand = reinterpret_cast<unsigned long long *>(base);
    base += align_up(sizeof(unsigned long long));
    e.CI = reinterpret_cast<int32_t *>(base);
    base += align_up((size_t)e.ccap * sizeof(int32_t));
    e.CJ = reinterpret_cast<int32_t *>(base);
    base += align_up((size_t)e.ccap * sizeof(int32_t));
    e.CV = reinterpret_cast<double *>(base);
    return e;
}

// The sketch (Compress) into R.  With nparts > 1 the inner index is split as
// planned by plan_sketch; before part c the stream waits for ready[c] (when
// given), so a producer on another stream may still be filling later parts.
int run_sketch(const void *A, int64_t lda, int transA, const void *B, int64_t ldb, int dtype,
               int64_t m, int64_t k, int64_t p, const cmm_hashes *hs, int prec, double *R,
               void *ws, cudaStream_t s, int nparts, const cudaEvent_t *ready, double ratio) {
    SketchPlan pl;
    plan_sketch(m, k, p, hs->d, hs->log2b, dtype, prec, transA, lda, ldb, pl, nparts, ratio);
    HashParams hp;
    fill_params(hs, hp);
    char *base = static_cast<char *>(ws);
    const size_t es = dtype_size(dtype);
    // bytes per element of the arrays the sketch reads: the workspace copies
    // (FP64 for the FP64 and fixed-point forms, else FP32) or the caller's
    const size_t tb = (prec == CMM_PREC_F64 || prec == CMM_PREC_FX64) ? 8 : 4;
    const size_t ea = pl.prep_A ? tb : dtype_size(dtype);
    const size_t eb = pl.prep_B ? tb : dtype_size(dtype);
    const int64_t b = int64_t(1) << hs->log2b;
    char *At = pl.prep_A ? base + pl.off_At : (char *)const_cast<void *>(A);
    char *Bp = pl.prep_B ? base + pl.off_Bp : (char *)const_cast<void *>(B);
    double *partial = reinterpret_cast<double *>(base + pl.off_partial);
    double *Z = reinterpret_cast<double *>(base + pl.off_Z);
    tab_t *tabA = reinterpret_cast<tab_t *>(base + pl.off_tab);
    tab_t *tabB = tabA + (size_t)hs->d * pl.C * m;
    float *colmax = reinterpret_cast<float *>(base + pl.off_colmax);
    cudaError_t e;
    if (pl.tmem) {
        Span sp("sketch_tables", s);
        e = launch_sketch_tm_tables(pl, m, p, hs->d, hp, tabA, tabB, s);
        if (e != cudaSuccess) return cuda_fail(e, "scatter tables");
    }
    int64_t blk0 = 0;
    for (int c = 0; c < pl.nparts; ++c) {
        const int64_t k0 = pl.kb[c], kp = pl.kb[c + 1] - pl.kb[c];
        if (ready && ready[c]) {
            e = cudaStreamWaitEvent(s, ready[c], 0);
            if (e != cudaSuccess) return cuda_fail(e, "wait for operand part");
        }
        // this part's column maxima (the per-column scales of the fixed-point
        // scatter): A^T rows, then B rows; taken by the preparation kernels
        // where they run, else by a pass over the caller's FP32 rows
        float *cm = colmax + 2 * k0;
        const bool fx = prec != CMM_PREC_F64 && prec != CMM_PREC_FX64 &&
                        prec != CMM_PREC_TERNARY && kp > 0;
        if (fx && (pl.prep_A || pl.prep_B)) {
            e = cudaMemsetAsync(cm, 0, 2 * kp * sizeof(float), s);
            if (e != cudaSuccess) return cuda_fail(e, "column maxima reset");
        }
        if (pl.prep_A && m > 0 && kp > 0) {
            Span sp("prep_A", s);
            // columns k0.. of A, or rows k0.. of A^T
            const char *Ap = static_cast<const char *>(A) + (transA ? k0 * lda : k0) * es;
            e = launch_prep_A(Ap, lda, transA, dtype, prec, m, kp, At + k0 * pl.ldat * tb, pl.ldat, s,
                              fx ? cm : nullptr);
            if (e != cudaSuccess) return cuda_fail(e, "prep A");
        }
        if (pl.prep_B && p > 0 && kp > 0) {
            Span sp("prep_B", s);
            e = launch_prep_B(static_cast<const char *>(B) + k0 * ldb * es, ldb, dtype, prec, kp, p,
                              Bp + k0 * pl.ldbp * tb, pl.ldbp, s, fx ? cm + kp : nullptr);
            if (e != cudaSuccess) return cuda_fail(e, "prep B");
        }
        const char *Atc = At + k0 * pl.ldat * ea;
        const char *Bpc = Bp + k0 * pl.ldbp * eb;
        if (fx && !(pl.prep_A && pl.prep_B)) {
            Span sp("colmax", s, (pl.prep_A || pl.prep_B) ? 1 : 2);
            e = cudaSuccess;
            if (!pl.prep_A) e = launch_rowmax((const float *)Atc, pl.ldat, kp, m, cm, s);
            if (e == cudaSuccess && !pl.prep_B)
                e = launch_rowmax((const float *)Bpc, pl.ldbp, kp, p, cm + kp, s);
            if (e != cudaSuccess) return cuda_fail(e, "column maxima");
        }
        SketchPlan pp = pl;   // this part's blocks
        pp.chunk = pl.pchunk[c];
        pp.nchunks = pl.pnch[c];
        double *pc = partial + blk0 * hs->d * b;
        blk0 += pl.pnch[c];
        if (prec == CMM_PREC_TERNARY) {
            // pack pairs of rows, check every entry, then sketch (one part)
            unsigned *Ap2 = reinterpret_cast<unsigned *>(base + pl.off_Ap2);
            unsigned *Bp2 = reinterpret_cast<unsigned *>(base + pl.off_Bp2);
            int *bad = reinterpret_cast<int *>(base + pl.off_bad);
            int hbad = 0;
            {
                Span sp("pack_pairs", s, 2);
                e = cudaMemsetAsync(bad, 0, sizeof(int), s);
                if (e == cudaSuccess)
                    e = launch_pack_pairs(Atc, ea == 8, pl.ldat, kp, m, reinterpret_cast<int *>(Ap2),
                                          bad, s);
                if (e == cudaSuccess)
                    e = launch_pack_pairs(Bpc, eb == 8, pl.ldbp, kp, p, reinterpret_cast<int *>(Bp2),
                                          bad, s);
            }
            if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(e, "ternary packing");
            if (hbad)
                return fail(CMM_ERR_ARG, "the ternary form needs every entry of A and B to be -1, 0 or 1");
            // int32 running sums: each pair adds at most 2 m p in magnitude
            const double mp2 = 2.0 * (double)std::max<int64_t>(m, 1) * (double)std::max<int64_t>(p, 1);
            const int flush = (int)std::max(1.0, std::floor(2147483647.0 / mp2));
            Span sp("sketch_ternary", s, 2);
            e = launch_sketch_i16(pp, Ap2, Bp2, m, (kp + 1) / 2, p, hs->d, hp, tabA, tabB, flush, pc, s);
        } else if (prec == CMM_PREC_FX64) {
            // quantise this part's rows of A^T and B to int64 fixed point, then sketch
            long long *Aq = reinterpret_cast<long long *>(base + pl.off_Aq) + k0 * m;
            long long *Bq = reinterpret_cast<long long *>(base + pl.off_Bq) + k0 * p;
            int *expA = reinterpret_cast<int *>(base + pl.off_exp) + k0;
            int *expB = reinterpret_cast<int *>(base + pl.off_exp) + k + k0;
            {
                Span sp("fx_quantize", s, 2);
                e = launch_fx_quantize((const double *)Atc, pl.ldat, kp, m, Aq, expA, s);
                if (e == cudaSuccess)
                    e = launch_fx_quantize((const double *)Bpc, pl.ldbp, kp, p, Bq, expB, s);
            }
            if (e != cudaSuccess) return cuda_fail(e, "fixed-point quantisation");
            Span sp("sketch_fx64", s, 2);
            e = launch_sketch_fx64(pp, Aq, Bq, m, kp, p, hs->d, hp, tabA, tabB, expA, expB, pc, s);
        } else if (pl.tmem) {
            Span sp("sketch_f32", s);
            e = launch_sketch_tm(pp, (const float *)Atc, (const float *)Bpc, m, kp, p, hs->d, tabA,
                                 tabB, cm, pc, s);
        } else {
            // these launchers build their scatter tables first (two launches)
            Span sp(prec == CMM_PREC_F64       ? "sketch_f64"
                    : prec == CMM_PREC_BF16TC ? "sketch_bf16tc"
                    : prec == CMM_PREC_F16TC  ? "sketch_f16tc"
                                              : "sketch_f32",
                    s, 2);
            if (prec == CMM_PREC_F64)
                e = launch_sketch_f64(pp, (const double *)Atc, (const double *)Bpc, m, kp, p,
                                      hs->d, hp, tabA, tabB, nullptr, pc, s);
            else if (prec_tc(prec))
                e = launch_sketch_bf16(pp, (const float *)Atc, (const float *)Bpc, m, kp, p, hs->d,
                                       hp, tabA, tabB, cm, pc, prec == CMM_PREC_F16TC, s);
            else
                e = launch_sketch_f32(pp, (const float *)Atc, (const float *)Bpc, m, kp, p, hs->d,
                                      hp, tabA, tabB, cm, pc, s);
        }
        if (e != cudaSuccess) return cuda_fail(e, "sketch kernel");
    }
    {
        Span sp("finish", s, 2);
        e = launch_finish(partial, pl.nchunks, hs->d, hs->log2b, Z, R, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "finish kernels");
    return CMM_OK;
}

// Decompress into C.  With hr non-null the estimates' heavy hitters are also
// collected on the way (launch_hh_cand writing C: counts and candidates per
// (row, tile) in the workspace) for finish_hh.
int run_extract(const double *R, const cmm_hashes *hs, int64_t m, int64_t p, int reduce,
                double *C, int64_t ldc, void *ws, cudaStream_t s, int cyclic, const HhRange *hr) {
    if (m == 0 || p == 0) return CMM_OK;
    HashParams hp;
    fill_params(hs, hp);
    ExtractWs ew = carve_extract(ws, m, p, hs->d);
    cudaError_t e;
    {
        Span sp("hash_tables", s);
        e = launch_hash_tables(hp, hs->d, hs->log2b, m, p, ew.H1, ew.H2, s);
    }
    if (e == cudaSuccess && hr) e = cudaMemsetAsync(ew.ncand, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "hash tables");
    {
        Span sp("extract", s);
        e = hr ? launch_hh_cand(R, ew.H1, ew.H2, hs->d, hs->log2b, m, p, m, 0, reduce, *hr, C, ldc,
                                ew.tcounts, ew.tsrc, ew.nt, ew.ncand, ew.ccap, ew.CI, ew.CJ,
                                ew.CV, s)
               : launch_extract(R, ew.H1, ew.H2, hs->d, hs->log2b, m, p, reduce, C, ldc, m, s,
                                cyclic);
    }
    if (e != cudaSuccess) return cuda_fail(e, "extract kernel");
    return CMM_OK;
}

// The heavy-hitter list of a dense C, given per-(row, tile) counts in
// ew.tcounts: row totals (and per row the tiles' inclusive prefix), a scan
// into offsets, then each row's hits in column order: copied from the
// candidates of launch_hh_cand when `cand` (read from C again for any tile
// whose candidates did not fit), else read from C by the tiles that hold
// them.  Rows past `capacity` are skipped on the device; one host
// synchronisation reads the total (and the candidate count).
int finish_hh(const ExtractWs &ew, bool cand, const double *C, int64_t ldc, int64_t m, int64_t p,
              HhRange hr, int32_t *I, int32_t *J, double *V, int64_t capacity, int64_t *count,
              cudaStream_t s) {
    cudaError_t e;
    {
        Span sp("hh_scan", s, 2);
        e = launch_hh_rowscan(ew.tcounts, ew.nt, m, p, ew.counts, s);
        if (e == cudaSuccess) e = launch_hh_scan(ew.counts, m, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "heavy-hitter scan");
    if (capacity > 0) {
        Span sp(cand ? "hh_copy" : "hh_write_dense", s);
        e = cand ? launch_hh_cand_copy(ew.tcounts, ew.tsrc, ew.nt, m, p, ew.counts + m, ew.CI,
                                       ew.CJ, ew.CV, ew.ccap, I, J, V, capacity, s)
                 : launch_hh_tile_write(C, ldc, m, p, hr, ew.tcounts, ew.nt, ew.counts + m, I, J,
                                        V, capacity, s);
        if (e != cudaSuccess) return cuda_fail(e, "heavy-hitter write");
    }
    int64_t total = 0;
    unsigned long long ncand = 0;
    e = cudaMemcpyAsync(&total, ew.counts + 2 * m, sizeof total, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && cand)
        e = cudaMemcpyAsync(&ncand, ew.ncand, sizeof ncand, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "heavy-hitter sync");
    if (cand && (int64_t)ncand > ew.ccap && capacity > 0) {
        {
            Span sp("hh_write_dense", s);
            e = launch_hh_tile_write(C, ldc, m, p, hr, ew.tcounts, ew.nt, ew.counts + m, I, J, V,
                                     capacity, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "heavy-hitter write");
    }
    *count = total;
    if (total > capacity)
        return fail(CMM_ERR_CAPACITY, "%lld heavy hitters, capacity %lld", (long long)total,
                    (long long)capacity);
    return CMM_OK;
}

// heavy hitters of the dense C
int run_hh_dense(const double *C, int64_t ldc, int64_t m, int64_t p, double tau, int32_t *I,
                 int32_t *J, double *V, int64_t capacity, int64_t *count, void *ws,
                 cudaStream_t s) {
    *count = 0;
    if (m == 0 || p == 0) return CMM_OK;
    ExtractWs ew = carve_extract(ws, m, p, 1);
    const HhRange hr = hh_range(tau);
    cudaError_t e;
    {
        Span sp("hh_count_dense", s);
        e = launch_hh_tile_count(C, ldc, m, p, hr, ew.tcounts, ew.nt, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "heavy-hitter count");
    return finish_hh(ew, false, C, ldc, m, p, hr, I, J, V, capacity, count, s);
}

// heavy hitters of the estimates from R, without writing C: one pass over the
// estimates writes the hits as candidates and counts them per (row, tile);
// row scan, scan, and the candidates are copied into order.  If there were
// more hits than candidate room, the list is written by a second pass that
// recomputes the estimates (the counts and offsets of the first stay valid).
int run_hh_R(const double *R, const cmm_hashes *hs, int64_t m, int64_t p, int reduce,
             double tau, int32_t *I, int32_t *J, double *V, int64_t capacity, int64_t *count,
             void *ws, cudaStream_t s) {
    *count = 0;
    if (m == 0 || p == 0) return CMM_OK;
    const int d = hs->d, L = hs->log2b;
    ExtractWs ew = carve_extract(ws, m, p, d);
    const HhRange hr = hh_range(tau);
    HashParams hp;
    fill_params(hs, hp);
    cudaError_t e;
    {
        Span sp("hash_tables", s);
        e = launch_hash_tables(hp, d, L, m, p, ew.H1, ew.H2, s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(ew.ncand, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "hash tables");
    {
        Span sp("hh_candidates", s);
        e = launch_hh_cand(R, ew.H1, ew.H2, d, L, m, p, m, 0, reduce, hr, nullptr, 0, ew.tcounts,
                           ew.tsrc, ew.nt, ew.ncand, ew.ccap, ew.CI, ew.CJ, ew.CV, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "heavy-hitter candidates");
    {
        Span sp("hh_scan", s, 2);
        e = launch_hh_rowscan(ew.tcounts, ew.nt, m, p, ew.counts, s);
        if (e == cudaSuccess) e = launch_hh_scan(ew.counts, m, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "heavy-hitter scan");
    if (capacity > 0) {
        Span sp("hh_copy", s);
        e = launch_hh_cand_copy(ew.tcounts, ew.tsrc, ew.nt, m, p, ew.counts + m, ew.CI, ew.CJ,
                                ew.CV, ew.ccap, I, J, V, capacity, s);
        if (e != cudaSuccess) return cuda_fail(e, "heavy-hitter copy");
    }
    int64_t total = 0;
    unsigned long long ncand = 0;
    e = cudaMemcpyAsync(&total, ew.counts + 2 * m, sizeof total, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&ncand, ew.ncand, sizeof ncand, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "heavy-hitter sync");
    if ((int64_t)ncand > ew.ccap && capacity > 0) {
        {
            Span sp("hh_write", s);
            e = launch_hh_write(R, ew.H1, ew.H2, d, L, m, p, reduce, hr, ew.counts + m, I, J, V,
                                capacity, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "heavy-hitter write");
    }
    *count = total;
    if (total > capacity)
        return fail(CMM_ERR_CAPACITY, "%lld heavy hitters, capacity %lld", (long long)total,
                    (long long)capacity);
    return CMM_OK;
}

}  // namespace api
}  // namespace cmm

int cmm::set_error(int code, const char *msg) { return api::fail(code, "%s", msg); }
