// cmm_internal.h -- declarations shared by the library's host code and its
// CUDA translation units (never by anything outside libcmm).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/cmm.h"

namespace cmm {

// Hash parameters of one repetition, passed by value in kernel parameters.
struct HashRep {
    uint64_t a1, c1;    // h1: rows of A -> buckets
    uint64_t a2, c2;    // h2: columns of B -> buckets
    uint64_t as1, cs1;  // s1: row signs
    uint64_t as2, cs2;  // s2: column signs
};

struct HashParams {
    HashRep rep[CMM_MAX_D];
};

// The heavy-hitter test abs(e) >= tau as an integer range on the magnitude
// bits of e (sign bit cleared): lo <= |bits(e)| <= hi.  tau <= 0 (either
// zero) gives [0, bits(+inf)], tau > 0 gives [bits(tau), bits(+inf)], and a
// NaN tau the empty range [1, 0]; NaN estimates lie above bits(+inf) and never
// pass, exactly as the FP64 comparison decides.  Integer compares keep the
// test off the FP64 pipe.
struct HhRange {
    unsigned long long lo, hi;
};
HhRange hh_range(double tau);

// One scatter-table word: padded shared-memory index of the bucket in the low
// 15 bits (slices of at most 2^14 points plus padding), the sign in bit 15.
using tab_t = uint16_t;

// Largest transform slice one CTA holds, per butterfly precision.
constexpr int kMaxLloF32 = 14;   // 2^14 FP32 = 64 KiB of shared memory
constexpr int kMaxLloF64 = 13;   // 2^13 FP64 = 64 KiB
constexpr int kMaxLloFx64 = 14;  // 2^14 int64 = 128 KiB (exact fixed-point form)
constexpr int kFinishLlo = 12;   // FP64 slice of the inverse transform: 2^12 doubles = 32 KiB

// Most parts a sketch is split into along the inner index (the host-buffer
// path sketches part c while part c + 1 is still being copied).
constexpr int kMaxParts = 4;

// Plan of one cmm_sketch call.
struct SketchPlan {
    int prec;              // CMM_PREC_*
    int L;                 // log2 b
    int Llo;               // log2 of the slice a CTA transforms
    int C;                 // 2^(L - Llo) slices per repetition
    int nchunks;           // blocks of the inner index
    int64_t chunk;         // inner indices per block (last may be shorter)
    int threads;           // CTA size
    size_t smem;           // dynamic shared memory per CTA
    // workspace carve-up (byte offsets into ws)
    size_t off_At, off_Bp, off_partial, off_Z, off_tab, off_colmax, total;
    // exact fixed-point form: int64 operands (k x m, k x p) and their row exponents (2k)
    size_t off_Aq, off_Bq, off_exp;
    // ternary form: packed pairs of rows (ceil(k/2) x m, ceil(k/2) x p words), the check word
    size_t off_Ap2, off_Bp2, off_bad;
    bool prep_A, prep_B;   // whether A / B are converted into the workspace
    int64_t ldat, ldbp;    // leading dimensions of the operands the sketch reads
    bool tmem;             // use the TMEM variant of the FP32 kernel
    // parts along the inner index: part c covers t in [kb[c], kb[c+1]) in
    // pnch[c] blocks of pchunk[c]; nchunks is the total, chunk part 0's
    int nclass;            // cyclic (FFT) form: frequency classes computed (C/2 + 1)
    int nparts;
    int64_t kb[kMaxParts + 1];
    int64_t pchunk[kMaxParts];
    int pnch[kMaxParts];
};

// Plan of one cmm_backward call (mean-estimator adjoint).
struct AdjointPlan {
    int prec, L, Llo, C, nchunks;
    int64_t chunk;
    int threads;
    size_t smem;
    bool prep_A, prep_B;
    int64_t ldat, ldbp;
    size_t off_At, off_Bp, off_G, off_Gs, off_Z, off_dAt, off_dBt, off_colmax, total;
    // FP32 with 2^14-point slices: the tensor-memory kernel (adjoint_tm.cu),
    // with the sketch's packed tables and an FP32 copy of Gs
    bool tm = false;
    size_t off_tabA = 0, off_tabB = 0, off_Gs32 = 0;
};

int adjoint_threads(int prec, int Llo);
cudaError_t launch_adj_g(const HashParams &hp, int d, int L, int64_t P, const int32_t *I,
                         const int32_t *J, const double *W, double *G, cudaStream_t s);
// colmax: the 2k column maxima of the FP32 fixed-point scatter (unused by FP64)
cudaError_t launch_adjoint(const AdjointPlan &pl, const void *At, const void *Bp, int64_t m,
                           int64_t k, int64_t p, int d, const HashParams &hp, const double *Gs,
                           const float *colmax, void *dAt, void *dBt, cudaStream_t s);
int adjoint_tm_threads();
int adjoint_tm_llo();
size_t adjoint_tm_smem(int64_t m, int64_t p);
cudaError_t launch_adjoint_tm(const AdjointPlan &pl, const float *At, const float *Bp, int64_t m,
                              int64_t k, int64_t p, int d, const HashParams &hp, const double *Gs,
                              float *Gs32, tab_t *tabA, tab_t *tabB, const float *colmax,
                              float *dAt, float *dBt, cudaStream_t s);
// dst (dst_dtype, leading dimension ldd) = src (rows x cols, FP64 when src_f64
// else FP32, contiguous), transposed when `transpose`
cudaError_t launch_convert_out(const void *src, int src_f64, int64_t rows, int64_t cols,
                               int transpose, void *dst, int dst_dtype, int64_t ldd,
                               cudaStream_t s);

// Record `msg` as the calling thread's cmm_last_error() text; returns `code`.
int set_error(int code, const char *msg);

// ---- launchers (prep.cu, sketch_f32.cu, sketch_f64.cu, sketch_tm.cu, sketch_bf16.cu, finish.cu) ----
// A^T (k x m) and B (k x p) in the butterfly type.  With FP32 output and rmax
// non-null, also rmax[t] = max(rmax[t], max |row t of the output|) (rmax
// zeroed by the caller): the row maxima of launch_rowmax without a second read.
cudaError_t launch_prep_A(const void *A, int64_t lda, int transA, int dtype, int prec,
                          int64_t m, int64_t k, void *At, int64_t ldat, cudaStream_t s,
                          float *rmax = nullptr);
cudaError_t launch_prep_B(const void *B, int64_t ldb, int dtype, int prec,
                          int64_t k, int64_t p, void *Bp, int64_t ldbp, cudaStream_t s,
                          float *rmax = nullptr);
// out[r] = max_c |X[r][c]| over the rows x cols FP32 array X (leading dimension
// ldx): the per-column scale of the fixed-point scatter
cudaError_t launch_rowmax(const float *X, int64_t ldx, int64_t rows, int64_t cols, float *out,
                          cudaStream_t s);
// tabA / tabB: scatter tables (d * C * m and d * C * p words, built by the
// launcher when not null); colmax: the 2k column maxima of the FP32
// fixed-point scatter (A^T rows, then B rows), unused by FP64
cudaError_t launch_sketch_f32(const SketchPlan &pl, const float *At, const float *Bp,
                              int64_t m, int64_t k, int64_t p, int d, const HashParams &hp,
                              const tab_t *tabA, const tab_t *tabB, const float *colmax,
                              double *partial, cudaStream_t s);
cudaError_t launch_sketch_f64(const SketchPlan &pl, const double *At, const double *Bp,
                              int64_t m, int64_t k, int64_t p, int d, const HashParams &hp,
                              const tab_t *tabA, const tab_t *tabB, const float *colmax,
                              double *partial, cudaStream_t s);
cudaError_t launch_finish(const double *partial, int nchunks, int d, int L, double *Z,
                          double *R, cudaStream_t s);
// TMEM variant of the FP32 sketch kernel (2^14-point slices)
bool sketch_tm_supported(int prec, int Llo);
int sketch_tm_threads();
size_t sketch_tm_smem();
// scatter tables of the TMEM kernel (d * C * m and d * C * p words)
cudaError_t launch_sketch_tm_tables(const SketchPlan &pl, int64_t m, int64_t p, int d,
                                    const HashParams &hp, tab_t *tabA, tab_t *tabB,
                                    cudaStream_t s);
// colmax: max |A[i][t]| over i for each t, then max |B[t][j]| over j (2k floats)
cudaError_t launch_sketch_tm(const SketchPlan &pl, const float *At, const float *Bp, int64_t m,
                             int64_t k, int64_t p, int d, const tab_t *tabA, const tab_t *tabB,
                             const float *colmax, double *partial, cudaStream_t s);
// 16-bit tensor-core variant (2^15-point slices, fixed-point scatter; colmax as
// for the FP32 kernels): BF16 operands, or FP16 operands with f16
int sketch_bf16_llo();
int sketch_bf16_threads();
size_t sketch_bf16_smem();
cudaError_t launch_sketch_bf16(const SketchPlan &pl, const float *At, const float *Bp, int64_t m,
                               int64_t k, int64_t p, int d, const HashParams &hp, tab_t *tabA,
                               tab_t *tabB, const float *colmax, double *partial, bool f16,
                               cudaStream_t s);
// cyclic (FFT) form of Sec. 3.1: 2^13-frequency classes, 32-bit tables of
// d * nclass * m and d * nclass * p words (built by the launcher), complex FP64
// partials [block][r][class][2^13][2]; the finish writes G [r][C][2^13][2]
int sketch_fft_llo();
int sketch_fft_threads();
size_t sketch_fft_smem();
cudaError_t launch_sketch_fft(const SketchPlan &pl, const float *At, const float *Bp, int64_t m,
                              int64_t k, int64_t p, int d, const HashParams &hp, uint32_t *tabA,
                              uint32_t *tabB, const float *colmax, double *partial,
                              cudaStream_t s);
cudaError_t launch_finish_fft(const double *partial, int nchunks, int d, int L, int C, int NC,
                              double *G, double *R, cudaStream_t s);
// exact 64-bit fixed-point form (CMM_PREC_FX64, sketch_fx64.cu): rows of X
// (k x n FP64, leading dimension ldx) quantised to Q (k x n int64) with one
// power of two 2^expo[t] per row (sum |Q[t][:]| < 2^62); the sketch kernel
// reads Q and the exponents and builds its own scatter tables (tabA, tabB)
int sketch_fx64_threads(int Llo);
size_t sketch_fx64_smem(int Llo);
cudaError_t launch_fx_quantize(const double *X, int64_t ldx, int64_t k, int64_t n, long long *Q,
                               int *expo, cudaStream_t s);
cudaError_t launch_sketch_fx64(const SketchPlan &pl, const long long *Aq, const long long *Bq,
                               int64_t m, int64_t k, int64_t p, int d, const HashParams &hp,
                               tab_t *tabA, tab_t *tabB, const int *expA, const int *expB,
                               double *partial, cudaStream_t s);
// exact form for ternary operands (CMM_PREC_TERNARY, sketch_i16.cu): rows of X
// (k x n, FP64 when x_f64 else FP32) packed in pairs, Wp[q][i] = X[2q][i] +
// 2^16 X[2q+1][i] (ceil(k/2) x n words); *bad |= 1 on an entry other than
// -1, 0, 1.  The sketch kernel builds its own tables; flush = pairs per int32
// running sum (2 m p flush < 2^31).
bool sketch_i16_supported(int Llo);
int sketch_i16_threads();
size_t sketch_i16_smem();
cudaError_t launch_pack_pairs(const void *X, int x_f64, int64_t ldx, int64_t k, int64_t n,
                              int *Wp, int *bad, cudaStream_t s);
cudaError_t launch_sketch_i16(const SketchPlan &pl, const unsigned *Ap, const unsigned *Bp,
                              int64_t m, int64_t npairs, int64_t p, int d, const HashParams &hp,
                              tab_t *tabA, tab_t *tabB, int flush, double *partial,
                              cudaStream_t s);
int sketch_threads_f32(int Llo);
int sketch_threads_f64(int Llo);
size_t sketch_smem_f32(int Llo);
size_t sketch_smem_f64(int Llo);

// ---- extraction (extract.cu) ----
cudaError_t launch_hash_tables(const HashParams &hp, int d, int L, int64_t m, int64_t p,
                               uint32_t *H1, uint32_t *H2, cudaStream_t s);
// rows [0, m) of C; H1 holds each repetition's row hashes at stride ldh (pass
// H1 + i0 and the full row count to extract rows i0 .. i0 + m - 1); cyclic
// selects the bucket (h1 + h2) mod b of Sec. 3.1 instead of h1 XOR h2
cudaError_t launch_extract(const double *R, const uint32_t *H1, const uint32_t *H2, int d,
                           int L, int64_t m, int64_t p, int reduce, double *C, int64_t ldc,
                           int64_t ldh, cudaStream_t s, int cyclic = 0);
int64_t hh_tiles(int64_t p);   // tiles of 256 columns per row: ceil(p / 256)
// exclusive scan of counts[0, n) into counts[n, 2n] (counts[2n] = total)
cudaError_t launch_hh_scan(int64_t *counts, int64_t n, cudaStream_t s);
// heavy hitters from R, estimates recomputed, at the offsets of a scan of the
// per-row counts (the second pass when the candidates of launch_hh_cand overflow)
cudaError_t launch_hh_write(const double *R, const uint32_t *H1, const uint32_t *H2, int d,
                            int L, int64_t m, int64_t p, int reduce, HhRange hr,
                            const int64_t *offsets, int32_t *I, int32_t *J, double *V,
                            int64_t capacity, cudaStream_t s);
// heavy hitters in one pass over the estimates of rows [0, m) (H1 at stride
// ldh as in launch_extract; row0 = the first row's index in the whole C):
// with C non-null the estimates are also written to C; the hits become
// candidates (ordered within each (row, tile of 256 columns)) at offsets of a
// counter, with their count and first offset per (row, tile); then, after
// the row scan and the scan of the row totals, the candidates are copied into
// the ordered list
cudaError_t launch_hh_cand(const double *R, const uint32_t *H1, const uint32_t *H2, int d, int L,
                           int64_t m, int64_t p, int64_t ldh, int64_t row0, int reduce, HhRange hr,
                           double *C, int64_t ldc, int32_t *tcounts, int64_t *tsrc, int64_t ldt,
                           unsigned long long *ncand, int64_t ccap, int32_t *CI, int32_t *CJ,
                           double *CV, cudaStream_t s);
cudaError_t launch_hh_cand_copy(const int32_t *tinc, const int64_t *tsrc, int64_t ldt, int64_t m,
                                int64_t p, const int64_t *offsets, const int32_t *CI,
                                const int32_t *CJ, const double *CV, int64_t ccap, int32_t *I,
                                int32_t *J, double *V, int64_t capacity, cudaStream_t s);
// heavy hitters of a dense m x p estimate C: hits per (row, tile) (the
// tiles of launch_hh_cand); per row, the tile counts turned in place
// into their inclusive prefix and the row total into counts[i]; then the
// ordered list, one warp per tile that holds hits
cudaError_t launch_hh_tile_count(const double *C, int64_t ldc, int64_t m, int64_t p, HhRange hr,
                                 int32_t *tcounts, int64_t ldt, cudaStream_t s);
cudaError_t launch_hh_rowscan(int32_t *tcounts, int64_t ldt, int64_t m, int64_t p,
                              int64_t *counts, cudaStream_t s);
cudaError_t launch_hh_tile_write(const double *C, int64_t ldc, int64_t m, int64_t p, HhRange hr,
                                 const int32_t *tinc, int64_t ldt, const int64_t *offsets,
                                 int32_t *I, int32_t *J, double *V, int64_t capacity,
                                 cudaStream_t s);
cudaError_t launch_mean_pairs(const double *R, const HashParams &hp, int d, int L, int64_t P,
                              const int32_t *I, const int32_t *J, double *out, cudaStream_t s);

}  // namespace cmm
