// host.cpp -- the C ABI of libcmm (include/cmm.h): argument checks, hash
// parameter generation, workspace planning and kernel launches.  No function
// here allocates device memory; every scratch byte comes from the caller's ws.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

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

// ---- launch tracing: CUDA events around every kernel launch while enabled ----
struct TraceRec {
    const char *name;
    int launches;
    cudaEvent_t a, b;
};
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

// RAII span: records an event on `s` at construction and at destruction
struct Span {
    bool on = false;
    TraceRec rec{};
    cudaStream_t s;
    Span(const char *name, cudaStream_t st, int launches = 1) : s(st) {
        std::lock_guard<std::mutex> lk(g_tr_mu);
        if (!g_tr_on) return;
        rec.name = name;
        rec.launches = launches;
        rec.a = tr_event();
        rec.b = tr_event();
        if (!rec.a || !rec.b) return;
        on = cudaEventRecord(rec.a, s) == cudaSuccess;
    }
    ~Span() {
        if (!on) return;
        cudaEventRecord(rec.b, s);
        std::lock_guard<std::mutex> lk(g_tr_mu);
        g_tr.push_back(rec);
    }
};

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
// nparts > 1 splits the inner index into parts (the host-buffer path): part
// c holds a share of k proportional to ratio^c (ratio <= 0: equal parts)
bool plan_sketch(int64_t m, int64_t k, int64_t p, int d, int L, int dtype, int prec, int transA,
                 int64_t lda, int64_t ldb, SketchPlan &pl, int nparts = 1,
                 double ratio = 0.0) {
    pl = SketchPlan{};
    pl.prec = prec;
    pl.L = L;
    const bool f64 = prec == CMM_PREC_F64;
    const bool bf16 = prec == CMM_PREC_BF16TC;
    if (bf16 && L < sketch_bf16_llo()) return false;
    const int maxLlo = bf16 ? sketch_bf16_llo() : (f64 ? kMaxLloF64 : kMaxLloF32);
    pl.Llo = std::min(L, maxLlo);
    pl.C = 1 << (L - pl.Llo);
    pl.tmem = sketch_tm_supported(prec, pl.Llo) && use_tmem_kernel();
    pl.threads = bf16 ? sketch_bf16_threads()
                      : pl.tmem ? sketch_tm_threads()
                                : (f64 ? sketch_threads_f64(pl.Llo) : sketch_threads_f32(pl.Llo));
    pl.smem = bf16 ? sketch_bf16_smem()
                   : pl.tmem ? sketch_tm_smem()
                             : (f64 ? sketch_smem_f64(pl.Llo) : sketch_smem_f32(pl.Llo));
    const int LE = bf16 ? pl.Llo : pl.tmem ? 7 : std::min(pl.Llo, f64 ? 4 : 5);
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
    if (k < nparts) nparts = 1;
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
        const int64_t kk = std::max<int64_t>(pl.kb[c + 1] - pl.kb[c], 1);
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
    pl.off_tab = off;
    off += align_up((size_t)d * pl.C * (m + p) * sizeof(tab_t));
    pl.off_colmax = off;
    if (prec != CMM_PREC_F64) off += align_up((size_t)2 * k * sizeof(float));
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

struct ExtractWs {
    uint32_t *H1, *H2;
    int64_t *counts;
    int32_t *tcounts;   // m x nt, row stride nt
    int64_t *tsrc;      // m x nt: offset of a (row, tile)'s first candidate
    int64_t nt;
    unsigned long long *ncand;
    int64_t ccap;
    int32_t *CI, *CJ;
    double *CV;
};

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
               void *ws, cudaStream_t s, int nparts = 1, const cudaEvent_t *ready = nullptr,
               double ratio = 0.0) {
    SketchPlan pl;
    plan_sketch(m, k, p, hs->d, hs->log2b, dtype, prec, transA, lda, ldb, pl, nparts, ratio);
    HashParams hp;
    fill_params(hs, hp);
    char *base = static_cast<char *>(ws);
    const size_t es = dtype_size(dtype);
    const size_t tb = prec == CMM_PREC_F64 ? 8 : 4;
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
        const bool fx = prec != CMM_PREC_F64 && kp > 0;
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
        const char *Atc = At + k0 * pl.ldat * tb;
        const char *Bpc = Bp + k0 * pl.ldbp * tb;
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
        if (pl.tmem) {
            Span sp("sketch_f32", s);
            e = launch_sketch_tm(pp, (const float *)Atc, (const float *)Bpc, m, kp, p, hs->d, tabA,
                                 tabB, cm, pc, s);
        } else {
            // these launchers build their scatter tables first (two launches)
            Span sp(prec == CMM_PREC_F64 ? "sketch_f64"
                    : prec == CMM_PREC_BF16TC ? "sketch_bf16tc" : "sketch_f32", s, 2);
            if (prec == CMM_PREC_F64)
                e = launch_sketch_f64(pp, (const double *)Atc, (const double *)Bpc, m, kp, p,
                                      hs->d, hp, tabA, tabB, nullptr, pc, s);
            else if (prec == CMM_PREC_BF16TC)
                e = launch_sketch_bf16(pp, (const float *)Atc, (const float *)Bpc, m, kp, p, hs->d,
                                       hp, tabA, tabB, cm, pc, s);
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
                double *C, int64_t ldc, void *ws, cudaStream_t s, int cyclic = 0,
                const HhRange *hr = nullptr) {
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
    if (pl.smem > kMaxDynSmem) return false;
    const int64_t slots = num_sms();
    const int64_t kk = std::max<int64_t>(k, 1);
    const int64_t nc_max = std::max<int64_t>(1, (kk + G - 1) / G);
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
    pl.total = off;
    return true;
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

int cmm::set_error(int code, const char *msg) { return fail(code, "%s", msg); }

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
    if (prec == CMM_PREC_BF16TC && hs->log2b < sketch_bf16_llo())
        return fail(CMM_ERR_RANGE, "precision BF16TC needs log2b >= %d", sketch_bf16_llo());
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
    if (prec == CMM_PREC_BF16TC && hs->log2b < sketch_bf16_llo())
        return fail(CMM_ERR_RANGE, "precision BF16TC needs log2b >= %d", sketch_bf16_llo());
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
    if (prec == CMM_PREC_BF16TC && hs->log2b < sketch_bf16_llo())
        return fail(CMM_ERR_RANGE, "precision BF16TC needs log2b >= %d", sketch_bf16_llo());
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
// operations (~18 Tops/s FP32, ~13 Tops/s BF16 blocks, ~0.45 Tops/s FP64).
// Kept within [1/2, 3]: only the first part's copy is exposed, and it shrinks
// as the later parts grow.
double host_part_ratio(int64_t m, int64_t p, int d, int L, size_t es, int prec) {
    const double b = std::ldexp(1.0, L);
    const double copy_t = (double)(m + p) * (double)es / 211e9;
    const double rate = prec == CMM_PREC_F64 ? 0.45e12 : prec == CMM_PREC_BF16TC ? 13e12 : 18e12;
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
    if (prec == CMM_PREC_BF16TC && hs->log2b < sketch_bf16_llo())
        return fail(CMM_ERR_RANGE, "precision BF16TC needs log2b >= %d", sketch_bf16_llo());
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
        Span sp(prec == CMM_PREC_F64 ? "adjoint_f64" : "adjoint_f32", s);
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
