// api_common.h -- helpers shared by the C ABI's translation units (api*.cpp):
// error text, launch tracing, argument checks, sketch / extraction planning
// and the host-side drivers of Compress, Decompress and the heavy-hitter
// lists.  Internal to libcmm.
#pragma once

#include <cstdarg>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "cmm_internal.h"

namespace cmm {
namespace api {

// the calling thread's cmm_last_error() text; fail() formats it and returns code
extern thread_local std::string g_err;
int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *where);

// ---- launch tracing: CUDA events around every kernel launch while enabled ----
struct TraceRec {
    const char *name;
    int launches;
    cudaEvent_t a, b;
};
extern std::mutex g_tr_mu;
extern bool g_tr_on;
extern std::vector<TraceRec> g_tr;
extern std::vector<cudaEvent_t> g_ev_pool;
cudaEvent_t tr_event();

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
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int num_sms();
int check_hashes(const cmm_hashes *hs);
void fill_params(const cmm_hashes *hs, HashParams &hp);
bool valid_dtype(int dt);
// the 16-bit tensor-core precisions (BF16 or FP16 operands)
inline bool prec_tc(int prec) { return prec == CMM_PREC_BF16TC || prec == CMM_PREC_F16TC; }
size_t dtype_size(int dt);
int check_sizes(int64_t m, int64_t k, int64_t p);
bool use_tmem_kernel();
int check_ws(void *ws, size_t ws_bytes, size_t need);
int check_prec_sizes(int prec, int log2b, int64_t m, int64_t p);
int check_operands(const void *A, int64_t lda, int transA, const void *B, int64_t ldb, int dtype,
                   int64_t m, int64_t k, int64_t p, int prec);

// nparts > 1 splits the inner index into parts (the host-buffer path): part
// c holds a share of k proportional to ratio^c (ratio <= 0: equal parts)
bool plan_sketch(int64_t m, int64_t k, int64_t p, int d, int L, int dtype, int prec, int transA,
                 int64_t lda, int64_t ldb, SketchPlan &pl, int nparts = 1, double ratio = 0.0);

// ---- extraction workspace ---------------------------------------------------
int64_t hh_cand_capacity(int64_t m, int64_t p);
size_t extract_ws_bytes(int64_t m, int64_t p, int d);
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
ExtractWs carve_extract(void *ws, int64_t m, int64_t p, int d);

// ---- drivers (stream-ordered; return CMM_OK or a CMM_ERR_* code) ------------
// Compress into R (d x b); with nparts > 1 the inner index is sketched in the
// parts plan_sketch(.., nparts, ratio) makes, part c after ready[c] is recorded
int run_sketch(const void *A, int64_t lda, int transA, const void *B, int64_t ldb, int dtype,
               int64_t m, int64_t k, int64_t p, const cmm_hashes *hs, int prec, double *R,
               void *ws, cudaStream_t s, int nparts = 1, const cudaEvent_t *ready = nullptr,
               double ratio = 0.0);
// Decompress into C; with hr the heavy hitters are collected on the way
int run_extract(const double *R, const cmm_hashes *hs, int64_t m, int64_t p, int reduce,
                double *C, int64_t ldc, void *ws, cudaStream_t s, int cyclic = 0,
                const HhRange *hr = nullptr);
// the ordered heavy-hitter list of a dense C from per-(row, tile) counts
// (candidates of launch_hh_cand when `cand`); synchronises s
int finish_hh(const ExtractWs &ew, bool cand, const double *C, int64_t ldc, int64_t m, int64_t p,
              HhRange hr, int32_t *I, int32_t *J, double *V, int64_t capacity, int64_t *count,
              cudaStream_t s);
int run_hh_dense(const double *C, int64_t ldc, int64_t m, int64_t p, double tau, int32_t *I,
                 int32_t *J, double *V, int64_t capacity, int64_t *count, void *ws,
                 cudaStream_t s);
int run_hh_R(const double *R, const cmm_hashes *hs, int64_t m, int64_t p, int reduce,
             double tau, int32_t *I, int32_t *J, double *V, int64_t capacity, int64_t *count,
             void *ws, cudaStream_t s);

}  // namespace api
}  // namespace cmm
