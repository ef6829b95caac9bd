/*
 * cmm_oracle.c -- plain, slow FP64 CPU oracle for compressed matrix multiplication
 * in its Fast Walsh-Hadamard Transform form (Andersson & Karppa, arXiv 2601.09477).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may link, load or call
 * this file: only the tests, the smoke check and the benchmark's CPU-baseline leg
 * do.  It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes, and where the paper defines it:
 *   - splitmix64 seed expansion (Steele, Lea & Flood 2014, the published
 *     reference generator) -> the 64-bit pairs (a, c) of every hash function.
 *     The paper only says "draw two random 64-bit integers" (Sec. 4.2); the
 *     seed -> (a, c) convention is this project's and is parity-pinned by the
 *     generator's published output plus agreement with the library.
 *   - multiply-add-shift hash h_{a,c}(x) = floor(((a*x + c) mod 2^64) / 2^(64-log2 b)),
 *     and the sign hash as the same family with b = 2 (Sec. 4.2); the sign is
 *     +1 when that top bit is 0 and -1 when it is 1.
 *   - the unnormalised Walsh-Hadamard transform in Sylvester (natural) order,
 *     H[u][v] = (-1)^popcount(u & v), as in-place butterflies (Sec. 3.2).
 *   - Compress (Algorithm 1): for every repetition r, for every inner index t,
 *     sketch column t of A and row t of B with (h1, s1) and (h2, s2), transform
 *     both, accumulate the pointwise product into p[r]; finally transform p[r].
 *     Algorithm 1 applies H three times without a scale; with the unnormalised H
 *     that gives b times the XOR convolution, so p[r] is scaled by 1/b at the
 *     end (reading of the normalisation stated in Sec. 3.2's identity).
 *   - Decompress (Algorithm 1): x_r = s1_r(i) s2_r(j) p[r][h1_r(i) XOR h2_r(j)],
 *     estimate = median over r (odd d: middle order statistic; even d: mean of
 *     the two middle values), or the mean over r for the differentiable form.
 *   - heavy hitters: all (i, j) with |estimate| >= tau, in row-major (i, j) order.
 *   - adjoint of the mean estimator at a list of pairs: the estimator is linear
 *     in C = A B, so the loss sum_q W_q Chat_mean[I_q, J_q] equals
 *     sum_{i,j} M[i][j] C[i][j] with
 *     M[i][j] = s1_r(i) s2_r(j) sum_r G_r[h1_r(i) XOR h2_r(j)],
 *     G_r[w]  = (1/d) sum_{q : h1_r(I_q) XOR h2_r(J_q) = w} W_q s1_r(I_q) s2_r(J_q),
 *     hence dL/dA = M B^T and dL/dB = A^T M (chain rule through C = A B).
 *
 * Indices are 0-based; hash keys are the 0-based row/column index (< 2^32).
 * Hash parameter layout, per repetition r, eight uint64 words:
 *   hp[8r+0..1] = (a, c) of h1,  hp[8r+2..3] = (a, c) of h2,
 *   hp[8r+4..5] = (a, c) of s1,  hp[8r+6..7] = (a, c) of s2.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- splitmix64 (Steele, Lea & Flood 2014) ------------------------------ */
static uint64_t orc_splitmix64_next(uint64_t *state)
{
    uint64_t z;
    *state += 0x9e3779b97f4a7c15ULL;
    z = *state;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* n successive outputs of splitmix64 started from `seed` */
void orc_splitmix64_stream(uint64_t seed, int64_t n, uint64_t *out)
{
    uint64_t s = seed;
    for (int64_t q = 0; q < n; ++q) out[q] = orc_splitmix64_next(&s);
}

/* Draw (a, c) for h1, h2, s1, s2 of d repetitions, in the order
 * a_h1, c_h1, a_h2, c_h2, a_s1, c_s1, a_s2, c_s2 per repetition. */
void orc_draw_hashes(uint64_t seed, int d, uint64_t *hp)
{
    orc_splitmix64_stream(seed, 8 * (int64_t)d, hp);
}

/* ---- hash family (Sec. 4.2) ----------------------------------------------- */
uint32_t orc_bucket(uint64_t a, uint64_t c, uint64_t x, int log2b)
{
    uint64_t v = a * x + c;                 /* arithmetic mod 2^64 */
    return (uint32_t)(v >> (64 - log2b));   /* the log2 b highest bits */
}

int orc_sign(uint64_t a, uint64_t c, uint64_t x)
{
    /* b = 2: the single highest bit; bit 0 -> +1, bit 1 -> -1 */
    return orc_bucket(a, c, x, 1) ? -1 : 1;
}

void orc_bucket_array(uint64_t a, uint64_t c, int64_t n, int log2b, uint32_t *out)
{
    for (int64_t x = 0; x < n; ++x) out[x] = orc_bucket(a, c, (uint64_t)x, log2b);
}

void orc_sign_array(uint64_t a, uint64_t c, int64_t n, int32_t *out)
{
    for (int64_t x = 0; x < n; ++x) out[x] = orc_sign(a, c, (uint64_t)x);
}

/* ---- Walsh-Hadamard transform, Sylvester order, unnormalised (Sec. 3.2) --- */
void orc_fwht(double *x, int log2b)
{
    int64_t b = (int64_t)1 << log2b;
    for (int64_t h = 1; h < b; h <<= 1)
        for (int64_t i = 0; i < b; i += 2 * h)
            for (int64_t j = i; j < i + h; ++j) {
                double u = x[j], v = x[j + h];
                x[j] = u + v;
                x[j + h] = u - v;
            }
}

/* element A[i][t] of the m x k left operand; transA = 1 means the array holds
 * A^T as a k x m row-major matrix (the paper's preferred layout, Sec. 4.3) */
static double orc_A(const double *A, int64_t lda, int transA, int64_t i, int64_t t)
{
    return transA ? A[t * lda + i] : A[i * lda + t];
}

/* ---- Compress (Algorithm 1) ------------------------------------------------
 * R is d x b row-major.  The loop over the inner index t is split across
 * `nthreads` OpenMP threads (each with its own accumulator, summed in thread
 * order at the end), which is the parallel-for over k of the paper's
 * implementation (Algorithm 2); nthreads = 1 is the literal serial order. */
int orc_compress(const double *A, int64_t lda, int transA,
                 const double *B, int64_t ldb,
                 int64_t m, int64_t k, int64_t p, int d, int log2b,
                 const uint64_t *hp, double *R, int nthreads)
{
    int64_t b = (int64_t)1 << log2b;
    if (nthreads < 1) nthreads = 1;
    for (int r = 0; r < d; ++r) {
        const uint64_t *q = hp + 8 * r;
        double *acc = (double *)calloc((size_t)nthreads * b, sizeof(double));
        if (!acc) return -1;
        int failed = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
        {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            double *pr = acc + (size_t)tid * b;
            double *pA = (double *)malloc(b * sizeof(double));
            double *pB = (double *)malloc(b * sizeof(double));
            if (!pA || !pB) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                failed = 1;
            } else {
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
                for (int64_t t = 0; t < k; ++t) {
                    memset(pA, 0, b * sizeof(double));          /* p_A <- 0_b */
                    for (int64_t i = 0; i < m; ++i)
                        pA[orc_bucket(q[0], q[1], (uint64_t)i, log2b)] +=
                            orc_sign(q[4], q[5], (uint64_t)i) * orc_A(A, lda, transA, i, t);
                    memset(pB, 0, b * sizeof(double));          /* p_B <- 0_b */
                    for (int64_t j = 0; j < p; ++j)
                        pB[orc_bucket(q[2], q[3], (uint64_t)j, log2b)] +=
                            orc_sign(q[6], q[7], (uint64_t)j) * B[t * ldb + j];
                    orc_fwht(pA, log2b);
                    orc_fwht(pB, log2b);
                    for (int64_t u = 0; u < b; ++u) pr[u] += pA[u] * pB[u];
                }
            }
            free(pA);
            free(pB);
        }
        if (failed) { free(acc); return -1; }
        double *Rr = R + (size_t)r * b;
        for (int64_t u = 0; u < b; ++u) {
            double s = 0.0;
            for (int th = 0; th < nthreads; ++th) s += acc[(size_t)th * b + u];
            Rr[u] = s;
        }
        free(acc);
        orc_fwht(Rr, log2b);                                   /* p[r] <- H{p[r]} */
        for (int64_t u = 0; u < b; ++u) Rr[u] /= (double)b;      /* 1/b normalisation */
    }
    return 0;
}

/* ---- Decompress (Algorithm 1) ---------------------------------------------- */
static void orc_sort(double *v, int n)
{
    for (int a = 1; a < n; ++a) {
        double key = v[a];
        int z = a - 1;
        while (z >= 0 && v[z] > key) { v[z + 1] = v[z]; --z; }
        v[z + 1] = key;
    }
}

/* reduce = 0: median; reduce = 1: mean */
double orc_decompress(const double *R, const uint64_t *hp, int d, int log2b,
                      int64_t i, int64_t j, int reduce)
{
    int64_t b = (int64_t)1 << log2b;
    double x[256];
    if (d < 1 || d > 256) return NAN;
    for (int r = 0; r < d; ++r) {
        const uint64_t *q = hp + 8 * r;
        uint32_t w = orc_bucket(q[0], q[1], (uint64_t)i, log2b) ^
                     orc_bucket(q[2], q[3], (uint64_t)j, log2b);
        x[r] = (double)(orc_sign(q[4], q[5], (uint64_t)i) * orc_sign(q[6], q[7], (uint64_t)j)) *
               R[(size_t)r * b + w];
    }
    if (reduce == 1) {
        double s = 0.0;
        for (int r = 0; r < d; ++r) s += x[r];
        return s / d;
    }
    orc_sort(x, d);
    if (d & 1) return x[d / 2];
    return 0.5 * (x[d / 2 - 1] + x[d / 2]);
}

/* full estimate, rows [i0, i1) of the m x p product, into C (ldc) */
void orc_decompress_rows(const double *R, const uint64_t *hp, int d, int log2b,
                         int64_t i0, int64_t i1, int64_t p, int reduce,
                         double *C, int64_t ldc, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (int64_t i = i0; i < i1; ++i)
        for (int64_t j = 0; j < p; ++j)
            C[(i - i0) * ldc + j] = orc_decompress(R, hp, d, log2b, i, j, reduce);
}

/* heavy hitters of rows [i0, i1): |estimate| >= tau in row-major order.
 * Writes at most `capacity` entries, returns the total number found. */
int64_t orc_heavy_hitters(const double *R, const uint64_t *hp, int d, int log2b,
                          int64_t i0, int64_t i1, int64_t p, int reduce, double tau,
                          int32_t *I, int32_t *J, double *V, int64_t capacity)
{
    int64_t n = 0;
    for (int64_t i = i0; i < i1; ++i)
        for (int64_t j = 0; j < p; ++j) {
            double e = orc_decompress(R, hp, d, log2b, i, j, reduce);
            if (fabs(e) >= tau) {
                if (n < capacity) { I[n] = (int32_t)i; J[n] = (int32_t)j; V[n] = e; }
                ++n;
            }
        }
    return n;
}

/* mean estimator at a list of P pairs */
void orc_mean_at_pairs(const double *R, const uint64_t *hp, int d, int log2b,
                       int64_t P, const int32_t *I, const int32_t *J, double *out)
{
    for (int64_t q = 0; q < P; ++q) out[q] = orc_decompress(R, hp, d, log2b, I[q], J[q], 1);
}

/* G_r[w] = (1/d) sum over pairs q with h1_r(I_q) XOR h2_r(J_q) = w of
 * W_q s1_r(I_q) s2_r(J_q);  G is d x b row-major */
void orc_adjoint_G(const uint64_t *hp, int d, int log2b, int64_t P,
                   const int32_t *I, const int32_t *J, const double *W, double *G)
{
    int64_t b = (int64_t)1 << log2b;
    memset(G, 0, (size_t)d * b * sizeof(double));
    for (int r = 0; r < d; ++r) {
        const uint64_t *q = hp + 8 * r;
        for (int64_t z = 0; z < P; ++z) {
            uint32_t w = orc_bucket(q[0], q[1], (uint64_t)I[z], log2b) ^
                         orc_bucket(q[2], q[3], (uint64_t)J[z], log2b);
            G[(size_t)r * b + w] += W[z] * orc_sign(q[4], q[5], (uint64_t)I[z]) *
                                    orc_sign(q[6], q[7], (uint64_t)J[z]) / (double)d;
        }
    }
}

/* rows [i0, i1) of M[i][j] = s1_r(i) s2_r(j) sum_r G_r[h1_r(i) XOR h2_r(j)]
 * (the sum over r includes the signs of that repetition) */
void orc_adjoint_M_rows(const double *G, const uint64_t *hp, int d, int log2b,
                        int64_t i0, int64_t i1, int64_t p, double *M, int64_t ldm)
{
    int64_t b = (int64_t)1 << log2b;
    for (int64_t i = i0; i < i1; ++i)
        for (int64_t j = 0; j < p; ++j) {
            double s = 0.0;
            for (int r = 0; r < d; ++r) {
                const uint64_t *q = hp + 8 * r;
                uint32_t w = orc_bucket(q[0], q[1], (uint64_t)i, log2b) ^
                             orc_bucket(q[2], q[3], (uint64_t)j, log2b);
                s += orc_sign(q[4], q[5], (uint64_t)i) * orc_sign(q[6], q[7], (uint64_t)j) *
                     G[(size_t)r * b + w];
            }
            M[(i - i0) * ldm + j] = s;
        }
}

/* One entry of the sketch straight from its definition (the bucketed product
 * that Compress reaches, Sec. 3.2 with Algorithm 1):
 *   R_r[w] = sum_{(i,j) : h1_r(i) XOR h2_r(j) = w} s1_r(i) s2_r(j) C[i][j],
 * C[i][j] = sum_t A[i][t] B[t][j], visiting every (i, j).  For sampled checks
 * of large problems where Compress itself would take too long on the CPU. */
double orc_R_entry(const double *A, int64_t lda, int transA, const double *B, int64_t ldb,
                   int64_t m, int64_t k, int64_t p, int log2b, const uint64_t *hp_r,
                   uint32_t w)
{
    double acc = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        uint32_t hi = orc_bucket(hp_r[0], hp_r[1], (uint64_t)i, log2b);
        int si = orc_sign(hp_r[4], hp_r[5], (uint64_t)i);
        for (int64_t j = 0; j < p; ++j) {
            if ((hi ^ orc_bucket(hp_r[2], hp_r[3], (uint64_t)j, log2b)) != w) continue;
            double c = 0.0;
            for (int64_t t = 0; t < k; ++t) c += orc_A(A, lda, transA, i, t) * B[t * ldb + j];
            acc += (double)(si * orc_sign(hp_r[6], hp_r[7], (uint64_t)j)) * c;
        }
    }
    return acc;
}

int orc_openmp_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
