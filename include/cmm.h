/*
 * cmm.h -- C ABI of libcmm, compressed matrix multiplication in the Fast
 * Walsh-Hadamard Transform form on one GB300 GPU (sm_103a).
 *
 * Method (Andersson & Karppa, "Engineering Compressed Matrix Multiplication
 * with the Fast Walsh-Hadamard Transform", arXiv 2601.09477, Algorithm 1):
 * for every repetition r < d, column t of A and row t of B are hashed into
 * signed sketches of length b = 2^log2b,
 *     x_t[u] = sum_{i : h1(i) = u} s1(i) A[i][t],   y_t[u] = sum_{j : h2(j) = u} s2(j) B[t][j],
 * transformed with the unnormalised Walsh-Hadamard matrix H[u][v] = (-1)^popcount(u & v),
 * multiplied pointwise and summed over t, then transformed back and scaled:
 *     R_r = (1/b) H sum_t (H x_t) o (H y_t)      (so R_r = sum_t x_t XOR-convolved with y_t).
 * The estimate of C = A B is Chat[i][j] = median_r s1_r(i) s2_r(j) R_r[h1_r(i) XOR h2_r(j)]
 * (Algorithm 1, Decompress).  The hashes are the multiply-add-shift family of
 * Sec. 4.2: h_{a,c}(x) = ((a x + c) mod 2^64) >> (64 - log2 b); a sign hash is
 * the same family with b = 2, +1 when that top bit is 0 and -1 when it is 1.
 *
 * Conventions for every entry point:
 *  - Matrices are row-major.  A is m x k (lda >= k) or, with transA = 1, the
 *    array holds A^T as k x m (lda >= m), the layout of Sec. 4.3.  B is k x p
 *    (ldb >= p).  Row/column indices are 0-based and are the hash keys, so
 *    m, p < 2^31.
 *  - Pointers named "device" are CUDA device (or managed) memory owned by the
 *    caller; the library never allocates or frees device memory.  Scratch space
 *    is the caller's `ws` buffer of at least the size the matching
 *    *_workspace_bytes query returns, 256-byte aligned.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls are asynchronous on that stream unless stated otherwise.
 *  - Argument errors are returned before anything is launched.  Every call
 *    returns a cmm_status; cmm_last_error() gives a message for the calling
 *    host thread.
 */
#ifndef CMM_H
#define CMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CMM_MAX_D 64        /* largest number of repetitions d */
#define CMM_MAX_LOG2B 24    /* largest sketch length b = 2^24 */

typedef enum {
    CMM_OK = 0,
    CMM_ERR_ARG = -1,        /* null pointer, negative size, bad enum, bad leading dimension */
    CMM_ERR_RANGE = -3,      /* size outside the supported range (d, log2b, m, p, k) */
    CMM_ERR_CAPACITY = -4,   /* heavy-hitter list longer than `capacity`; *count is the true size */
    CMM_ERR_CUDA = -5,       /* a CUDA runtime call or launch failed */
    CMM_ERR_TIMEOUT = -6,    /* a bounded device-side wait ran out (batched launch) */
    CMM_ERR_WORKSPACE = -8   /* ws is NULL, misaligned or smaller than the query returned */
} cmm_status;

/* storage type of A and B */
typedef enum { CMM_F64 = 0, CMM_F32 = 1, CMM_BF16 = 2 } cmm_dtype;

/* arithmetic of the sketch transforms and the per-block multiply-accumulate.
 * The cross-block reduction of R over t, the inverse transform and the
 * extraction are FP64 in every precision. */
typedef enum {
    CMM_PREC_F64 = 0,     /* FP64 butterflies and accumulation ("plain FP64") */
    CMM_PREC_F32 = 1,     /* FP32 butterflies, FP32 accumulation within a block of t */
    CMM_PREC_BF16TC = 2,  /* BF16 operands with exact +-1 Hadamard blocks on the tensor cores, FP32 accumulation */
    CMM_PREC_F16TC = 3,   /* as BF16TC with FP16 operands, scaled to a fixed range (3 more significand bits) */
    CMM_PREC_FX64 = 4,    /* exact 64-bit fixed-point butterflies: each column quantised once to integers
                           * with sum |q| < 2^62 (per-column power of two from its l1 norm), scatter and
                           * transforms exact in int64, float-float multiply-accumulate; R within the
                           * FP64 tolerance (quantisation <= 2^-60 |column|_1 per value).  Operands must
                           * be finite. */
    CMM_PREC_TERNARY = 5  /* exact integer form for operands whose entries are all -1, 0 or +1 (the
                           * +-1 inputs of Sec. 5.2): two inner indices per pass as one 32-bit word of
                           * two 16-bit halves, int32 multiply-accumulate into an int64 sum, R exact.
                           * Needs log2b >= 14 and m, p < 2^15 (else CMM_ERR_RANGE); any other entry
                           * gives CMM_ERR_ARG, found by a check that synchronises the stream. */
} cmm_prec;

/* how the d repetitions are combined */
typedef enum { CMM_MEDIAN = 0, CMM_MEAN = 1 } cmm_reduce;

/* Hash functions of all repetitions (Sec. 4.2).  `params` is a HOST array of
 * 8*d words; for repetition r the words 8r .. 8r+7 are
 *   a, c of h1 (rows of A -> buckets),  a, c of h2 (columns of B -> buckets),
 *   a, c of s1 (row signs),             a, c of s2 (column signs).
 * The library copies them into kernel parameters; the array may be freed after
 * the call returns. */
typedef struct {
    int32_t d;               /* repetitions, 1 .. CMM_MAX_D */
    int32_t log2b;           /* sketch length b = 2^log2b, 1 .. CMM_MAX_LOG2B */
    const uint64_t *params;  /* host, 8*d words */
} cmm_hashes;

/* Fill `params` (host, 8*d words) from a 64-bit seed with splitmix64
 * (Steele, Lea & Flood 2014): the words are its successive outputs in the
 * order of cmm_hashes.params.  The paper draws (a, c) as "two random 64-bit
 * integers" (Sec. 4.2) and fixes no generator; this one is the library's
 * convention.  Errors: CMM_ERR_ARG (params NULL), CMM_ERR_RANGE (d). */
int cmm_make_hashes(uint64_t seed, int32_t d, uint64_t *params);

/* Bytes of `ws` needed by cmm_sketch for these sizes (0 on invalid sizes). */
size_t cmm_sketch_workspace_bytes(int64_t m, int64_t k, int64_t p, int32_t d, int32_t log2b,
                                  int32_t dtype, int32_t prec, int32_t transA);

/* Compress (Algorithm 1): R (device, d x b FP64, row-major) = the sketch of
 * A B for every repetition, already scaled by 1/b, i.e.
 *   R_r[w] = sum_{(i,j) : h1_r(i) XOR h2_r(j) = w} s1_r(i) s2_r(j) (A B)[i][j]
 * up to the rounding of the chosen precision.  A, B: device, `dtype`.
 * k = 0 gives R = 0.  Errors: CMM_ERR_ARG, CMM_ERR_RANGE, CMM_ERR_WORKSPACE,
 * CMM_ERR_CUDA. */
int cmm_sketch(const void *A, int64_t lda, int32_t transA, const void *B, int64_t ldb,
               int32_t dtype, int64_t m, int64_t k, int64_t p, const cmm_hashes *hs,
               int32_t prec, double *R, void *ws, size_t ws_bytes, void *stream);

/* Size of the static scratch array used by cmm_sketch_noalloc (64 MiB). */
#define CMM_SKETCH_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)

/* cmm_sketch for callers that cannot allocate device memory (the paper has no
 * counterpart: its CPU code allocates freely).  Such callers include serving
 * processes that reserve their whole device-memory budget at start-up, plugins
 * whose host application owns every device allocation, and latency-critical
 * paths that cannot take cudaMalloc's implicit synchronisation.  Same
 * arguments and result as cmm_sketch, without `ws`: the scratch is a static
 * device array of CMM_SKETCH_NOALLOC_SCRATCH_BYTES in the library, held by
 * every GPU that loads the library until the process exits.  A problem whose
 * cmm_sketch_workspace_bytes exceeds that size is rejected with CMM_ERR_RANGE
 * before anything runs.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current and keeps it
 * for the CUDA context it was found in; a call in another context, or after a
 * cudaDeviceReset, finds a new context id and looks the address up again.
 * Make the first call on each device (and the first after a reset) before any
 * stream capture.  All calls share the array, so calls that overlap on the GPU
 * race and must be serialised by the caller.  The function calls no
 * cudaMalloc/cudaFree or other allocating routine. */
int cmm_sketch_noalloc(const void *A, int64_t lda, int32_t transA, const void *B, int64_t ldb,
                       int32_t dtype, int64_t m, int64_t k, int64_t p, const cmm_hashes *hs,
                       int32_t prec, double *R, void *stream);

/* Bytes of `ws` needed by cmm_extract / cmm_heavy_hitters / cmm_threshold. */
size_t cmm_extract_workspace_bytes(int64_t m, int64_t p, int32_t d);

/* Decompress (Algorithm 1) for every entry: C (device, m x p FP64, ldc >= p)
 *   C[i][j] = reduce_r s1_r(i) s2_r(j) R_r[h1_r(i) XOR h2_r(j)]
 * with reduce = median (middle order statistic for odd d, mean of the two
 * middle values for even d) or mean.  R: device, d x b FP64 from cmm_sketch.
 * Errors: CMM_ERR_ARG, CMM_ERR_RANGE, CMM_ERR_WORKSPACE, CMM_ERR_CUDA. */
int cmm_extract(const double *R, const cmm_hashes *hs, int64_t m, int64_t p, int32_t reduce,
                double *C, int64_t ldc, void *ws, size_t ws_bytes, void *stream);

/* Heavy hitters straight from the sketch (the goal of the method, Sec. 1):
 * every (i, j) with |Chat[i][j]| >= tau, sorted by (i, j) row-major, written to
 * I, J (device int32) and V (device FP64, the estimate) up to `capacity`
 * entries, without writing Chat: one pass over the estimates (a second when
 * there are more hits than one per 64 entries).  *count (HOST) receives the
 * total number found.  Synchronises `stream` to read the count.  Returns
 * CMM_ERR_CAPACITY when *count > capacity (the first `capacity` entries are
 * still written). */
int cmm_heavy_hitters(const double *R, const cmm_hashes *hs, int64_t m, int64_t p,
                      int32_t reduce, double tau, int32_t *I, int32_t *J, double *V,
                      int64_t capacity, int64_t *count, void *ws, size_t ws_bytes,
                      void *stream);

/* The same list from a dense estimate C (device, m x p FP64, ldc): entries
 * with |C[i][j]| >= tau in (i, j) order.  Same outputs and errors as
 * cmm_heavy_hitters. */
int cmm_threshold(const double *C, int64_t m, int64_t p, int64_t ldc, double tau,
                  int32_t *I, int32_t *J, double *V, int64_t capacity, int64_t *count,
                  void *ws, size_t ws_bytes, void *stream);

/* Bytes of `ws` needed by cmm_multiply. */
size_t cmm_multiply_workspace_bytes(int64_t m, int64_t k, int64_t p, int32_t d, int32_t log2b,
                                    int32_t dtype, int32_t prec, int32_t transA);

/* Compress then Decompress every entry: C (device, m x p FP64) = the estimate
 * of A B.  R (device, d x b FP64) receives the sketch; it may be NULL, in
 * which case the sketch lives in `ws`.  Errors: as cmm_sketch and cmm_extract. */
int cmm_multiply(const void *A, int64_t lda, int32_t transA, const void *B, int64_t ldb,
                 int32_t dtype, int64_t m, int64_t k, int64_t p, const cmm_hashes *hs,
                 int32_t prec, int32_t reduce, double *C, int64_t ldc, double *R,
                 void *ws, size_t ws_bytes, void *stream);

/* cmm_multiply followed by cmm_threshold(C, tau) in one call (Algorithm 1's
 * Decompress, then the goal of Sec. 1): the heavy hitters are collected while
 * Decompress writes C, so the list costs no further pass over C (one pass
 * when there are more hits than one per 64 entries of C).  Outputs as
 * cmm_multiply (C, R) plus the list of cmm_threshold: I, J (device int32), V
 * (device FP64), `capacity` entries, *count (HOST) = total found.
 * Synchronises `stream` to read the count.  `ws`:
 * cmm_multiply_workspace_bytes.  Errors: as cmm_multiply, plus
 * CMM_ERR_CAPACITY as in cmm_threshold. */
int cmm_multiply_threshold(const void *A, int64_t lda, int32_t transA, const void *B,
                           int64_t ldb, int32_t dtype, int64_t m, int64_t k, int64_t p,
                           const cmm_hashes *hs, int32_t prec, int32_t reduce, double *C,
                           int64_t ldc, double *R, double tau, int32_t *I, int32_t *J,
                           double *V, int64_t capacity, int64_t *count, void *ws,
                           size_t ws_bytes, void *stream);

/* ---- Pagh's original cyclic form (Sec. 3.1), through the FFT --------------
 * The paper's comparison form: the same sketches x_t, y_t and hash functions,
 * but the product polynomial is the cyclic convolution of Sec. 2, so
 *   R_r[w] = sum_{(i,j) : (h1_r(i) + h2_r(j)) mod b = w} s1_r(i) s2_r(j) (A B)[i][j],
 * computed as R_r = (1/b) IDFT( sum_t DFT(x_t) o DFT(y_t) ).  The forward
 * transforms and the products run in FP32 (complex, 2^13-frequency slices);
 * the reduction over t, the inverse transform and the extraction are FP64.
 * prec must be CMM_PREC_F32 (else CMM_ERR_ARG) and log2b >= 13 (else
 * CMM_ERR_RANGE); arguments, layouts, ownership and the other errors are those
 * of cmm_sketch. */
size_t cmm_sketch_cyclic_workspace_bytes(int64_t m, int64_t k, int64_t p, int32_t d,
                                         int32_t log2b, int32_t dtype, int32_t prec,
                                         int32_t transA);
int cmm_sketch_cyclic(const void *A, int64_t lda, int32_t transA, const void *B, int64_t ldb,
                      int32_t dtype, int64_t m, int64_t k, int64_t p, const cmm_hashes *hs,
                      int32_t prec, double *R, void *ws, size_t ws_bytes, void *stream);

/* Decompress of the cyclic form for every entry:
 *   C[i][j] = reduce_r s1_r(i) s2_r(j) R_r[(h1_r(i) + h2_r(j)) mod b]
 * (R from cmm_sketch_cyclic; `ws` of cmm_extract_workspace_bytes); otherwise
 * as cmm_extract.  Heavy hitters of the cyclic estimate: cmm_threshold. */
int cmm_extract_cyclic(const double *R, const cmm_hashes *hs, int64_t m, int64_t p,
                       int32_t reduce, double *C, int64_t ldc, void *ws, size_t ws_bytes,
                       void *stream);

/* cmm_sketch_cyclic then cmm_extract_cyclic (as cmm_multiply). */
size_t cmm_multiply_cyclic_workspace_bytes(int64_t m, int64_t k, int64_t p, int32_t d,
                                           int32_t log2b, int32_t dtype, int32_t prec,
                                           int32_t transA);
int cmm_multiply_cyclic(const void *A, int64_t lda, int32_t transA, const void *B,
                        int64_t ldb, int32_t dtype, int64_t m, int64_t k, int64_t p,
                        const cmm_hashes *hs, int32_t prec, int32_t reduce, double *C,
                        int64_t ldc, double *R, void *ws, size_t ws_bytes, void *stream);

/* Bytes of `ws` (device) needed by cmm_multiply_host with room for a
 * heavy-hitter list of `capacity` entries. */
size_t cmm_multiply_host_workspace_bytes(int64_t m, int64_t k, int64_t p, int32_t d,
                                         int32_t log2b, int32_t dtype, int32_t prec,
                                         int32_t transA, int64_t capacity);

/* cmm_multiply for operands in HOST memory (pinned memory gives full copy
 * speed; pageable memory works too): A and B (host, `dtype`, leading
 * dimensions as in cmm_sketch) are copied into `ws`, the estimate is computed
 * there, C (host, m x p FP64, ldc >= p; may be NULL) receives it, and when
 * `count` is not NULL the heavy hitters |C[i][j]| >= tau in (i, j) order are
 * copied to I, J, V (host, `capacity` entries; *count = total found).
 * Synchronous: returns once the results are in host memory.  Errors: as
 * cmm_multiply, plus CMM_ERR_CAPACITY as in cmm_threshold. */
int cmm_multiply_host(const void *A, int64_t lda, int32_t transA, const void *B, int64_t ldb,
                      int32_t dtype, int64_t m, int64_t k, int64_t p, const cmm_hashes *hs,
                      int32_t prec, int32_t reduce, double *C, int64_t ldc, double tau,
                      int64_t capacity, int32_t *I, int32_t *J, double *V, int64_t *count,
                      void *ws, size_t ws_bytes, void *stream);

/* Mean estimator at a list of P pairs (the differentiable form):
 * out[q] = (1/d) sum_r s1_r(I[q]) s2_r(J[q]) R_r[h1_r(I[q]) XOR h2_r(J[q])].
 * I, J: device int32 (0 <= I < m, 0 <= J < p, not checked on the device);
 * out: device FP64.  The paper has no mean form; it is the unbiased
 * single-repetition estimator of Sec. 3.1 averaged over r.
 * Errors: CMM_ERR_ARG, CMM_ERR_RANGE, CMM_ERR_CUDA. */
int cmm_mean_pairs(const double *R, const cmm_hashes *hs, int64_t P, const int32_t *I,
                   const int32_t *J, double *out, void *stream);

/* Bytes of `ws` needed by cmm_backward (0 on invalid sizes, or when m + p is
 * too large for the per-CTA gradient row and column in shared memory). */
size_t cmm_backward_workspace_bytes(int64_t m, int64_t k, int64_t p, int32_t d, int32_t log2b,
                                    int32_t dtype, int32_t prec, int32_t transA);

/* Adjoint of the mean estimator (cmm_mean_pairs) for the loss
 *   L(A, B) = sum_q W[q] * Chat_mean[I[q]][J[q]].
 * The estimator is bilinear in (A, B) (it is linear in C = A B through the
 * bucketed sketch of Algorithm 1), so with
 *   G_r[w] = (1/d) sum_{q : h1_r(I_q) XOR h2_r(J_q) = w} W_q s1_r(I_q) s2_r(J_q)
 * the gradients are
 *   dA[i][t] = s1_r(i) sum_r (G_r XOR-conv y_{r,t})[h1_r(i)],
 *   dB[t][j] = s2_r(j) sum_r (G_r XOR-conv x_{r,t})[h2_r(j)],
 * each XOR convolution computed as (1/b) H((H G_r) o (H y)) (Sec. 3.2).  The
 * paper has no gradient; this is the chain rule through its Compress.
 * A, B: device, FP32 or FP64 (dtype), layouts as in cmm_sketch.  I, J: device
 * int32 (P pairs); W: device FP64.  dA (device, A's dtype and layout: m x k,
 * or k x m when transA; leading dimension ldda) and dB (device, k x p, lddb)
 * are overwritten.  prec: CMM_PREC_F64 or CMM_PREC_F32 (butterflies).
 * Errors: CMM_ERR_ARG, CMM_ERR_RANGE (m + p too large), CMM_ERR_WORKSPACE,
 * CMM_ERR_CUDA. */
int cmm_backward(const void *A, int64_t lda, int32_t transA, const void *B, int64_t ldb,
                 int32_t dtype, int64_t m, int64_t k, int64_t p, const cmm_hashes *hs,
                 int32_t prec, int64_t P, const int32_t *I, const int32_t *J, const double *W,
                 void *dA, int64_t ldda, void *dB, int64_t lddb, void *ws, size_t ws_bytes,
                 void *stream);

/* ---- many independent problems in one persistent launch ------------------
 * Each problem runs the whole path of Algorithm 1 (Compress and Decompress of
 * every entry) with its own sizes, sketch length and hash functions; the
 * repetition count d is shared.  The paper runs one problem at a time; this
 * batched form is the library's own. */
typedef struct {
    const void *A;                 /* device, A^T stored k x m row-major (transA must be 1) */
    int64_t lda;                   /* >= m */
    int32_t transA;                /* must be 1: the left operand transposed (Sec. 4.3) */
    const void *B;                 /* device, k x p row-major */
    int64_t ldb;                   /* >= p */
    int64_t m, k, p;
    int32_t log2b;                 /* 5 .. CMM_MAX_LOG2B */
    const uint64_t *hash_params;   /* host, 8*d words as in cmm_hashes.params */
    double *R;                     /* device out, d x 2^log2b FP64 */
    double *C;                     /* device out, m x p FP64 (NULL: sketch only) */
    int64_t ldc;                   /* >= p when C is set */
    int32_t tile_log2;             /* b-tile: log2 of the slice one CTA transforms, 0 = default */
    int64_t t_tile;                /* t-tile: inner indices per sketch task, 0 = default */
} cmm_problem;

/* Host-side handle filled by cmm_batched_prepare (no device memory). */
typedef struct {
    uint64_t opaque[32];
} cmm_batch_plan;

/* Bytes of `ws` for a batch (0 on invalid problems).  Supported: dtype
 * CMM_F32, prec CMM_PREC_F32. */
size_t cmm_batched_workspace_bytes(const cmm_problem *problems, int32_t Q, int32_t d,
                                   int32_t dtype, int32_t prec);

/* Validate the Q problems (host array), lay out `ws` and upload the task
 * table, problem descriptors and hash functions into it; synchronises
 * `stream`.  The operand and output pointers are recorded: later launches read
 * and write the same buffers.  Errors: CMM_ERR_ARG, CMM_ERR_RANGE,
 * CMM_ERR_WORKSPACE, CMM_ERR_CUDA. */
int cmm_batched_prepare(const cmm_problem *problems, int32_t Q, int32_t d, int32_t dtype,
                        int32_t prec, void *ws, size_t ws_bytes, cmm_batch_plan *plan,
                        void *stream);

/* One run of every problem: a memset of the task counters and ONE persistent
 * kernel launch on `stream`, both capturable in a CUDA graph.  Asynchronous. */
int cmm_batched_launch(const cmm_batch_plan *plan, void *stream);

/* cmm_batched_launch with explicit wait settings: `wait_budget_us` bounds
 * every dependency wait inside the kernel (0 = the default of about 4 s), and
 * a nonzero `unmet_dependency` raises each finish task's dependency target by
 * one so that no wait can be met -- the kernel then gives up after the
 * budget, sets its error word and returns, which lets a test exercise the
 * CMM_ERR_TIMEOUT path without faulting or hanging the GPU. */
int cmm_batched_launch_opts(const cmm_batch_plan *plan, int64_t wait_budget_us,
                            int32_t unmet_dependency, void *stream);

/* Synchronise `stream` and report whether the last launch finished:
 * CMM_ERR_TIMEOUT when a bounded dependency wait inside the kernel ran out. */
int cmm_batched_status(const cmm_batch_plan *plan, void *stream);

/* Launch tracing (the library's profiling hook).  While enabled, every
 * kernel launch the library makes is bracketed by CUDA events recorded on the
 * caller's stream.  cmm_trace_enable(1) clears earlier records and starts
 * recording; cmm_trace_enable(0) stops.  cmm_trace_read waits for the recorded
 * events and returns, per kernel name (at most max_entries of them, each name a
 * NUL-terminated string in a 32-byte slot of `names`, host), the number of
 * launches and the summed device time in ms; *n_out (host) is the number of
 * distinct names.  Tracing adds two event records per launch.  The paper has
 * no counterpart (it reports wall-clock times only, Sec. 5.4). */
int cmm_trace_enable(int32_t on);
int cmm_trace_read(int32_t max_entries, char *names, int64_t *launches, double *total_ms,
                   int32_t *n_out);

/* Last error message of the calling host thread ("" when none). */
const char *cmm_last_error(void);

/* Library version string. */
const char *cmm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CMM_H */
