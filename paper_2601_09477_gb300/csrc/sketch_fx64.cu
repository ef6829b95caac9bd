// sketch_fx64.cu -- the sketch (Algorithm 1's loop over the inner index t)
// with exact 64-bit fixed-point butterflies: results within the FP64
// tolerance of the plain FP64 form, without running the butterflies on the
// FP64 pipe (which this GPU issues at 1/64 of the FP32 rate).
//
// Fixed point.  Column t of A (row t of A^T) is quantised once, before the
// sketch, as q_i = round(a_i 2^e) with one power of two per column chosen
// from its l1 norm so that sum_i |q_i| <= 2^61 + m/2 < 2^62.  Every bucket sum
// of the scatter and every value of the Walsh-Hadamard transform of a slice is
// then an exact integer of magnitude below 2^62 (|H f|_inf <= |f|_1 <= sum_i
// |q_i|), so the scatter and all butterflies are exact int64 arithmetic and
// independent of the order of the atomics.  The only rounding before the
// multiply is the quantisation, |a_i - q_i 2^-e| <= 2^-(e+1) <= 2^-61 |a|_1
// (2^-60 |a|_1 when |a|_1 lies just below a power of two, see the bound
// below), which moves R_r[w] by at most 2^-60 c_max (|A_t|_1 |B_t|_1 + ...)
// per t -- about 2^-44 of sum_t |A_t|_2 |B_t|_2 at m = p = 8192 in the worst case.
//
// Multiply-accumulate.  Each transformed value X^ (int64) is split into three
// 21-bit chunks that convert to FP32 exactly (a magic-number add, no
// conversion instruction: this GPU converts 64-bit integers at the FP64 rate)
// and summed error-free into a float-float pair (xh, xl) with xh + xl = X^ to
// 2^-48.  Products X^ Y^ are formed error-free (FMA) and accumulated over the
// block of t in float-float (TwoSum), ~2^-46 relative; the block's sum is
// written as an FP64 partial and the cross-block reduction, the inverse
// transform and the extraction are FP64 as in every form.
//
// Work decomposition as in the other sketch kernels: one CTA = (repetition r,
// frequency slice u_hi of 2^14 points, block of t); 512 threads, 32 int64
// values per thread in three register rounds (5 + 5 + 4 index bits); the
// slice's int64 values are two 32-bit arrays in shared memory (low and high
// halves, 2 x 72 KiB padded, so that the scatter's atomics spread over all 32
// banks and round 0 reads 16-byte vectors), X^ and the running sum Z as
// float-float in tensor memory (4 words per point, all 512 columns), one CTA
// per SM.  (Slices of 2^13 with two CTAs of 256 threads per SM scatter every
// column twice as often: 31.0 against 27.0 ms at n = 8192, b = 2^16, d = 9.)  Scatter: each int64 is added to shared memory as two 32-bit
// atomics, the low word's carry-out (from the returned old value) added into
// the high word, which sums the 64-bit values exactly in any order (a 64-bit
// shared atomic add runs ~6x slower here).
#include "cmm_internal.h"
#include "fwht_device.cuh"
#include "sketch_impl.cuh"
#include "tmem_device.cuh"

namespace cmm {

namespace {

// ---------------------------------------------------------------- quantisation
// One CTA per row t of X (k rows of n FP64 values, leading dimension ldx):
// an upper bound U of l1 = sum |X[t][:]|, e[t] = 61 - E with U < 2^E, and
// Q[t][i] = round(X[t][i] 2^e) (int64, leading dimension n; the scaling is a
// shift of the significand, so e may leave the FP64 exponent range, as it does
// for columns of norm below 2^-962).  The bound is taken in integers on the bits of the entries (an FP64
// add runs at 1/64 of the FP32 rate here, and the sum of n FP64 adds per row
// made this kernel FP64-bound): with emax the largest binary exponent of a
// nonzero entry, each entry's significand is cut to at most 31 bits at
// emax's scale and the cuts plus one per entry are summed in 64 bits, so
// l1 <= U <= l1 (1 + n 2^-30) in those units: E is l1's own exponent unless
// l1 lies within that factor below a power of two (then e is one smaller, a
// quantisation step of 2^-60 instead of 2^-61 of l1).  Integer maxima and
// sums do not depend on their order: e is reproducible run to run.
constexpr int kQThreads = 256;

// round(a 2^e) for |a 2^e| < 2^62, with integer operations on the bits of a
// (a conversion instruction from FP64 runs at the FP64 rate here): a =
// mant 2^(ex - 1075), so a 2^e = mant 2^sh with sh = ex - 1075 + e; halves
// round away from zero
__device__ __forceinline__ long long quantize_bits(double a, int e) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
    const int ex = (int)((bits >> 52) & 0x7ff);
    unsigned long long mant = bits & 0xFFFFFFFFFFFFFull;
    if (ex) mant |= 1ull << 52;
    const int sh = (ex ? ex : 1) - 1075 + e;
    unsigned long long q;
    if (sh >= 0)   // subnormal entries of a column of tiny norm: |a 2^e| < 2^62 bounds the shift
        q = sh < 64 ? mant << sh : 0ull;
    else if (sh > -64)
        q = (mant + (1ull << (-sh - 1))) >> (-sh);
    else
        q = 0ull;
    return (bits >> 63) ? -(long long)q : (long long)q;
}

// rows are read in batches of kQBatch entries per thread, all loads first
constexpr int kQBatch = 8;

__global__ void __launch_bounds__(kQThreads)
fx_quantize_kernel(const double *__restrict__ X, int64_t ldx, int64_t k, int64_t n,
                   long long *__restrict__ Q, int *__restrict__ expo) {
    __shared__ int s_max[kQThreads / 32];
    __shared__ unsigned long long s_sum[kQThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr unsigned long long kM52 = 0xFFFFFFFFFFFFFull;
    constexpr int64_t kStep = (int64_t)kQBatch * kQThreads;
    for (int64_t t = blockIdx.x; t < k; t += gridDim.x) {
        const unsigned long long *row = reinterpret_cast<const unsigned long long *>(X + t * ldx);
        // the largest binary exponent field of a nonzero entry (1 for subnormals)
        int mx = 0;
        for (int64_t i0 = tid; i0 < n; i0 += kStep) {
            unsigned long long b[kQBatch];
#pragma unroll
            for (int u = 0; u < kQBatch; ++u) {
                const int64_t i = i0 + (int64_t)u * kQThreads;
                b[u] = i < n ? row[i] : 0ull;
            }
#pragma unroll
            for (int u = 0; u < kQBatch; ++u) {
                const int ex = (int)((b[u] >> 52) & 0x7ff);
                if (b[u] << 1) mx = max(mx, ex ? ex : 1);
            }
        }
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (lane == 0) s_max[warp] = mx;
        __syncthreads();
        int emax = 0;
#pragma unroll
        for (int w = 0; w < kQThreads / 32; ++w) emax = max(emax, s_max[w]);
        int e = 0;
        if (emax > 0) {
            // sum over the entries of floor(significand / 2^(emax - exponent + 22)) + 1
            unsigned long long S = 0;
            for (int64_t i0 = tid; i0 < n; i0 += kStep) {
                unsigned long long b[kQBatch];
#pragma unroll
                for (int u = 0; u < kQBatch; ++u) {
                    const int64_t i = i0 + (int64_t)u * kQThreads;
                    b[u] = i < n ? row[i] : 0ull;
                }
#pragma unroll
                for (int u = 0; u < kQBatch; ++u) {
                    if (b[u] << 1) {
                        const int ex = (int)((b[u] >> 52) & 0x7ff);
                        const unsigned long long mant = (b[u] & kM52) | (ex ? 1ull << 52 : 0ull);
                        const int sh = emax - (ex ? ex : 1) + 22;
                        S += (sh < 64 ? mant >> sh : 0ull) + 1ull;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
            if (lane == 0) s_sum[warp] = S;
            __syncthreads();
            unsigned long long U = 0;
#pragma unroll
            for (int w = 0; w < kQThreads / 32; ++w) U += s_sum[w];
            // l1 < U 2^(emax - 1075 + 22) <= 2^E
            const int E = (64 - __clzll((long long)U)) + emax - 1053;
            e = 61 - E;   // within [-995, 1112] for finite entries: 2^e need not be a double
        }
        __syncthreads();   // s_max and s_sum are reused by the next row
        long long *qrow = Q + t * n;
        const double *xr = X + t * ldx;
        for (int64_t i0 = tid; i0 < n; i0 += kStep) {
            double a[kQBatch];
#pragma unroll
            for (int u = 0; u < kQBatch; ++u) {
                const int64_t i = i0 + (int64_t)u * kQThreads;
                a[u] = i < n ? xr[i] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < kQBatch; ++u) {
                const int64_t i = i0 + (int64_t)u * kQThreads;
                if (i < n) qrow[i] = quantize_bits(a[u], e);
            }
        }
        if (tid == 0) expo[t] = e;
    }
}

}  // namespace

cudaError_t launch_fx_quantize(const double *X, int64_t ldx, int64_t k, int64_t n, long long *Q,
                               int *expo, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    const int64_t g = k < 152 * 8 ? k : 152 * 8;
    fx_quantize_kernel<<<(unsigned)g, kQThreads, 0, s>>>(X, ldx, k, n, Q, expo);
    return cudaGetLastError();
}

}  // namespace cmm

namespace cmm {

namespace {

// ---------------------------------------------------------------- device helpers
// 2^ex as a float; 0 below the normal range (such terms are negligible: see
// the block scale in sketch_fx64_kernel)
__device__ __forceinline__ float pow2f(int ex) {
    return ex < -126 ? 0.f : __int_as_float((127 + (ex > 127 ? 127 : ex)) << 23);
}

// c * s exactly, for |c| < 2^22 and s a power of two (or 0): 1.5 2^23 + c is
// exact in FP32 (its unit in the last place is 1), so (that - 1.5 2^23) * s
// is formed by one FMA without rounding
__device__ __forceinline__ float chunk_f(int c, float s) {
    const float mf = __int_as_float(0x4B400000 + c);
    return __fmaf_rn(mf, s, -12582912.f * s);
}

// v (int64, |v| < 2^63) times 2^ex as a float-float pair h + l: three 21-bit
// chunks, each exact in FP32; the top two are summed error-free (Fast2Sum:
// the top chunk's term is 0 or larger than the middle one's) and the bottom
// chunk is added to the error term
__device__ __forceinline__ void to_ff(long long v, int ex, float &h, float &l) {
    const int c2 = (int)(v >> 42);                                  // signed, |c2| <= 2^21
    const int c1 = (int)((unsigned long long)v >> 21) & 0x1FFFFF;   // 0 .. 2^21 - 1
    const int c0 = (int)v & 0x1FFFFF;
    const float a = chunk_f(c2, pow2f(ex + 42));
    const float b = chunk_f(c1, pow2f(ex + 21));
    const float c = chunk_f(c0, pow2f(ex));
    const float s = a + b;
    const float e = b - (s - a);
    h = s;
    l = e + c;
}

// (zh, zl) += (xh + xl)(yh + yl): the product error-free to ~2^-46, the sum
// by TwoSum with the errors gathered in zl
__device__ __forceinline__ void ff_mac(float xh, float xl, float yh, float yl, float &zh,
                                       float &zl) {
    const float ph = xh * yh;
    const float pe = __fmaf_rn(xh, yh, -ph);
    const float pl = __fmaf_rn(xh, yl, __fmaf_rn(xl, yh, pe));
    const float s = zh + ph;
    const float bb = s - zh;
    const float err = (zh - (s - bb)) + (ph - bb);
    zl = zl + (err + pl);
    zh = s;
}

// to_ff and ff_mac on two values at once with packed FP32x2 instructions
// (identical results: each lane is an IEEE operation of its own)
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// FP32 values with the bit patterns w0, w1 of floats in [2^23, 2^24) (unit
// in the last place 1), minus `base`, times s: exact for the chunks below
__device__ __forceinline__ float2 chunk_f2(uint32_t w0, uint32_t w1, float base, float s) {
    const float2 mf = make_float2(__uint_as_float(w0), __uint_as_float(w1));
    const float2 ss = make_float2(s, s);
    const float2 k = make_float2(-base * s, -base * s);
    return __ffma2_rn(mf, ss, k);
}

// the chunk bit patterns: the low and middle 21-bit chunks are OR-ed into the
// mantissa of 2^23 (one logic operation each: 2^23 + c), the signed top chunk
// (|c2| < 2^20 for |v| < 2^62) is offset by 2^21 (2^23 + 2^21 + c2)
__device__ __forceinline__ uint32_t top_bits(long long v) {
    return (uint32_t)((int)(v >> 42) + 0x4B200000);
}
__device__ __forceinline__ uint32_t mid_bits(long long v) {
    return ((uint32_t)((unsigned long long)v >> 21) & 0x1FFFFFu) | 0x4B000000u;
}
__device__ __forceinline__ uint32_t low_bits(long long v) {
    return ((uint32_t)v & 0x1FFFFFu) | 0x4B000000u;
}

__device__ __forceinline__ void to_ff2(long long v0, long long v1, float s42, float s21,
                                       float s0, float2 &h, float2 &l) {
    const float2 a = chunk_f2(top_bits(v0), top_bits(v1), 10485760.f, s42);   // 2^23 + 2^21
    const float2 b = chunk_f2(mid_bits(v0), mid_bits(v1), 8388608.f, s21);    // 2^23
    const float2 c = chunk_f2(low_bits(v0), low_bits(v1), 8388608.f, s0);
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 sm = __fadd2_rn(a, b);
    const float2 e = __ffma2_rn(__ffma2_rn(a, m1, sm), m1, b);   // b - (s - a)
    h = sm;
    l = __fadd2_rn(e, c);
}

__device__ __forceinline__ void ff_mac2(float2 xh, float2 xl, float2 yh, float2 yl, float2 &zh,
                                        float2 &zl) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 ph = __fmul2_rn(xh, yh);
    const float2 pe = __ffma2_rn(xh, yh, neg2(ph));
    const float2 pl = __ffma2_rn(xh, yl, __ffma2_rn(xl, yh, pe));
    const float2 sm = __fadd2_rn(zh, ph);
    const float2 bb = __ffma2_rn(zh, m1, sm);                     // s - zh
    const float2 e1 = __ffma2_rn(__ffma2_rn(bb, m1, sm), m1, zh); // zh - (s - bb)
    const float2 e2 = __ffma2_rn(bb, m1, ph);                     // ph - bb
    zl = __fadd2_rn(zl, __fadd2_rn(__fadd2_rn(e1, e2), pl));
    zh = sm;
}

// scatter one fixed-point column (n int64 values) with the packed table
// (padded word of the bucket in bits 0-14, sign in bit 15).  Each int64 is
// added to the slice (two 32-bit arrays, low and high halves) by two 32-bit
// atomics: the low word's carry-out, read from the old value it returns, goes
// into the high word with the value's high half, so the 64-bit sums are exact
// in any order.  Batches of B values per thread: all loads first, then the
// low-word atomics of four values at a time (their round trips overlap;
// eight at a time spill registers), then those values' high words.
template <int P, int B = 8>
__device__ __forceinline__ void scatter_batch(unsigned *lo, int *hi, const long long (&v)[B],
                                              const tab_t (&w)[B], int cnt) {
    constexpr int H = B < 4 ? B : 4;   // low-word atomics in flight at once
#pragma unroll
    for (int e0 = 0; e0 < B; e0 += H) {
        unsigned old[H];
#pragma unroll
        for (int e = 0; e < H; ++e) {
            const long long s = (w[e0 + e] >> 15) ? -v[e0 + e] : v[e0 + e];
            if (e0 + e < cnt) old[e] = atomicAdd(lo + (w[e0 + e] & 0x7fffu), (unsigned)s);
        }
#pragma unroll
        for (int e = 0; e < H; ++e) {
            if (e0 + e < cnt) {
                const long long s = (w[e0 + e] >> 15) ? -v[e0 + e] : v[e0 + e];
                const unsigned l = (unsigned)s;
                const int h = (int)(s >> 32) + ((old[e] + l) < old[e] ? 1 : 0);
                if (h != 0) atomicAdd(hi + (w[e0 + e] & 0x7fffu), h);
            }
        }
    }
}

template <int P, int B = 8>
__device__ __forceinline__ void scatter_fx(unsigned *lo, int *hi, const long long *__restrict__ col,
                                           const tab_t *__restrict__ tab, int64_t n, int q) {
    int64_t i = q;
    for (; i + (B - 1) * (int64_t)P < n; i += B * (int64_t)P) {
        long long v[B];
        tab_t w[B];
#pragma unroll
        for (int e = 0; e < B; ++e) {
            v[e] = __ldcs(col + i + e * (int64_t)P);
            w[e] = __ldg(tab + i + e * (int64_t)P);
        }
        scatter_batch<P, B>(lo, hi, v, w, B);
    }
    if (i < n) {
        long long v[B];
        tab_t w[B];
#pragma unroll
        for (int e = 0; e < B; ++e) {
            const bool ok = i + e * (int64_t)P < n;
            v[e] = ok ? __ldcs(col + i + e * (int64_t)P) : 0ll;
            w[e] = ok ? __ldg(tab + i + e * (int64_t)P) : (tab_t)0;
        }
        // the elements of the last batch are the first (n - i + P - 1) / P of it
        scatter_batch<P, B>(lo, hi, v, w, (int)((n - i + P - 1) / P));
    }
}


// The 2^L-point transform of a group's slice held as two 32-bit arrays (low
// and high halves of the int64 values, the padded FP32 word layout of
// fwht_device.cuh), leaving the result in v (last-round layout) and the
// arrays zeroed for the next scatter.  Round 0 reads its contiguous rows as
// 16-byte vectors; the last round (of two or more) reads each word and zeroes
// it by one exchange, so no clearing pass is needed, and ends with the
// group's barrier before its butterflies (the arrays are free from there on).
template <int L, int LE, int K>
__device__ __forceinline__ void fx_rounds(int *lo, int *hi, long long (&v)[1 << LE], int q,
                                          int g) {
    using S = FwhtShape<float, L, LE>;
    using RK = typename S::template Round<K>;
    constexpr int E = S::E;
    constexpr bool kVec = K == 0 && S::PAD == 4;
    constexpr bool kExch = K > 0 && K + 1 == S::NR;
    int *bl = lo + RK::addr(q, 0);
    int *bh = hi + RK::addr(q, 0);
    if constexpr (kVec) {
#pragma unroll
        for (int c = 0; c < E / 4; ++c) {
            const int4 a = reinterpret_cast<const int4 *>(bl)[c];
            const int4 b = reinterpret_cast<const int4 *>(bh)[c];
            v[4 * c] = (long long)(((unsigned long long)(unsigned)b.x << 32) | (unsigned)a.x);
            v[4 * c + 1] = (long long)(((unsigned long long)(unsigned)b.y << 32) | (unsigned)a.y);
            v[4 * c + 2] = (long long)(((unsigned long long)(unsigned)b.z << 32) | (unsigned)a.z);
            v[4 * c + 3] = (long long)(((unsigned long long)(unsigned)b.w << 32) | (unsigned)a.w);
        }
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int o = RK::addr(0, j);
            const unsigned a = kExch ? (unsigned)atomicExch(bl + o, 0) : (unsigned)bl[o];
            const unsigned b = kExch ? (unsigned)atomicExch(bh + o, 0) : (unsigned)bh[o];
            v[j] = (long long)(((unsigned long long)b << 32) | a);
        }
        // every read of the slice is done: the group's next scatter may start
        // while this round's butterflies and the caller's conversion run
        if constexpr (kExch) group_sync<S::P>(g);
    }
    reg_fwht_r4<long long, E, RK::nb>(v);
    if constexpr (K + 1 < S::NR) {
        if constexpr (kVec) {
#pragma unroll
            for (int c = 0; c < E / 4; ++c) {
                reinterpret_cast<int4 *>(bl)[c] =
                    make_int4((int)v[4 * c], (int)v[4 * c + 1], (int)v[4 * c + 2], (int)v[4 * c + 3]);
                reinterpret_cast<int4 *>(bh)[c] =
                    make_int4((int)(v[4 * c] >> 32), (int)(v[4 * c + 1] >> 32),
                              (int)(v[4 * c + 2] >> 32), (int)(v[4 * c + 3] >> 32));
            }
        } else {
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const int o = RK::addr(0, j);
                bl[o] = (int)v[j];
                bh[o] = (int)(v[j] >> 32);
            }
        }
        group_sync<S::P>(g);
        fx_rounds<L, LE, K + 1>(lo, hi, v, q, g);
    } else if constexpr (!kExch) {
        // a single round: zero the words it read
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int o = RK::addr(0, j);
            bl[o] = 0;
            bh[o] = 0;
        }
    }
}

// ---------------------------------------------------------------- the sketch kernel
template <int L>
struct FxCfg {
    // 2^14-point slices: one CTA of 512 threads per SM (147 KB of shared
    // memory, all 512 TMEM columns); smaller slices: 256 threads, 2 CTAs/SM
    static constexpr int THREADS = L == 14 ? 512 : 256;
    static constexpr int MINB = THREADS == 512 ? 1 : 2;
    static constexpr int LE = L < 5 ? L : 5;
    using S = FwhtShape<float, L, LE>;   // 32-bit word layout of each half array
    static constexpr int E = S::E, P = S::P, G = THREADS / P;
    static constexpr bool TM = LE == 5;   // X^ and Z in tensor memory (else registers)
    static constexpr uint32_t COLS = THREADS / 128 * 128;   // 4 words per point per thread
    static constexpr size_t SMEM = (size_t)2 * G * S::STRIDE * sizeof(int);   // low, high
    static_assert(THREADS % P == 0, "CTA must hold whole groups");
    static_assert((size_t)S::N * sizeof(double) <= SMEM, "FP64 reduction must fit");
};

// One CTA: repetition r, slice u_hi, inner indices [t0, t1) of the block.
// Aq / Bq: fixed-point operands (k x m, k x p int64), expA / expB their
// per-row exponents; tables as for the FP32 kernels (int64 word layout).
template <int L>
__global__ void __launch_bounds__(FxCfg<L>::THREADS, FxCfg<L>::MINB)
sketch_fx64_kernel(const long long *__restrict__ Aq, const long long *__restrict__ Bq,
                   int64_t m, int64_t k, int64_t p, int Lfull, int C, int64_t chunk, int d,
                   const tab_t *__restrict__ tabA, const tab_t *__restrict__ tabB,
                   const int *__restrict__ expA, const int *__restrict__ expB,
                   double *__restrict__ partial) {
    using Cfg = FxCfg<L>;
    using S = typename Cfg::S;
    constexpr int E = Cfg::E, P = Cfg::P, G = Cfg::G, LE = Cfg::LE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t s_taddr;
    constexpr int kFxThreads = Cfg::THREADS;
    __shared__ int s_red[kFxThreads / 32];

    int item = blockIdx.x;
    const uint32_t u_hi = (uint32_t)(item % C);
    item /= C;
    const int r = item % d;
    const int64_t blk = item / d;
    const int64_t t0 = blk * chunk;
    const int64_t t1 = (t0 + chunk < k) ? t0 + chunk : k;
    const int64_t b = (int64_t)1 << Lfull;
    const int64_t slot = (int64_t)r * C + u_hi;
    const tab_t *tA = tabA + slot * m;
    const tab_t *tB = tabB + slot * p;
    double *out = partial + (blk * d + r) * b + (int64_t)u_hi * S::N;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = tid / P, q = tid % P;
    int *sm = reinterpret_cast<int *>(smem_raw);
    int *lo = sm + g * S::STRIDE;              // low halves of the group's slice
    int *hi = sm + (G + g) * S::STRIDE;        // high halves

    if constexpr (Cfg::TM) {
        if (warp == 0) tm::alloc(&s_taddr, Cfg::COLS);
    }
    for (int i = tid; i < 2 * G * S::STRIDE; i += kFxThreads) sm[i] = 0;

    // block scale: S_ref = max over the block's t of 64 - eA_t - eB_t
    int mx = -0x40000000;
    for (int64_t t = t0 + tid; t < t1; t += kFxThreads) mx = max(mx, 64 - expA[t] - expB[t]);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((tid & 31) == 0) s_red[warp] = mx;
    if constexpr (Cfg::TM) tm::fence_before();
    __syncthreads();
    if constexpr (Cfg::TM) tm::fence_after();
    int sref = s_red[0];
#pragma unroll
    for (int w = 1; w < kFxThreads / 32; ++w) sref = max(sref, s_red[w]);
    if (t1 <= t0) sref = 0;

    // this thread's TMEM columns: lane 32 (warp mod 4) + lane id, column block
    // 128 (warp / 4): xh [0, E), xl [E, 2E), zh [2E, 3E), zl [3E, 4E)
    uint32_t tcol = 0;
    float xr[2 * E], zr[2 * E];   // register copies when the slice is small
    if constexpr (Cfg::TM) {
        tcol = s_taddr + ((uint32_t)(32 * (warp & 3)) << 16) + 128u * (uint32_t)(warp >> 2);
        uint32_t zero[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) zero[e] = 0u;
#pragma unroll
        for (int c = 0; c < 2 * E / 16; ++c) tm::st16(tcol + 2 * E + 16 * c, zero);
        tm::wait_st();
    } else {
#pragma unroll
        for (int j = 0; j < 2 * E; ++j) zr[j] = 0.f;
    }

    long long v[E];
    const int64_t nt = t1 > t0 ? t1 - t0 : 0;
    const int64_t iters = (nt + G - 1) / G;   // the same trip count for every group
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t t = t0 + it * G + g;
        const bool active = t < t1;
        // A's values carry the block scale 2^(64 - eA - eB - S_ref) <= 1 and
        // 2^-32 (keeps the float-float products and sums in range)
        const int exA = active ? (64 - expA[t] - expB[t] - sref) - 32 : -1000;
        const float sA42 = pow2f(exA + 42), sA21 = pow2f(exA + 21), sA0 = pow2f(exA);
        if (active) {
            // 16 elements in flight per thread when every thread has at least
            // that many, else 8 (a mostly empty batch costs more than it hides)
            if (m >= 16 * P)
                scatter_fx<P, 16>(reinterpret_cast<unsigned *>(lo), hi, Aq + t * m, tA, m, q);
            else
                scatter_fx<P, 8>(reinterpret_cast<unsigned *>(lo), hi, Aq + t * m, tA, m, q);
        }
        group_sync<P>(g);
        fx_rounds<L, LE, 0>(lo, hi, v, q, g);
        if constexpr (Cfg::TM) {
#pragma unroll
            for (int c = 0; c < E / 16; ++c) {
                uint32_t hw[16], lw[16];
#pragma unroll
                for (int e = 0; e < 16; e += 2) {
                    float2 h, l;
                    to_ff2(v[16 * c + e], v[16 * c + e + 1], sA42, sA21, sA0, h, l);
                    hw[e] = __float_as_uint(h.x);
                    hw[e + 1] = __float_as_uint(h.y);
                    lw[e] = __float_as_uint(l.x);
                    lw[e + 1] = __float_as_uint(l.y);
                }
                tm::st16(tcol + 16 * c, hw);
                tm::st16(tcol + E + 16 * c, lw);
            }
        } else {
#pragma unroll
            for (int j = 0; j < E; ++j) to_ff(v[j], exA, xr[j], xr[E + j]);
        }
        if constexpr (S::NR < 2) group_sync<P>(g);   // else synchronised in the last round
        if (active) {
            if (p >= 16 * P)
                scatter_fx<P, 16>(reinterpret_cast<unsigned *>(lo), hi, Bq + t * p, tB, p, q);
            else
                scatter_fx<P, 8>(reinterpret_cast<unsigned *>(lo), hi, Bq + t * p, tB, p, q);
        }
        group_sync<P>(g);
        fx_rounds<L, LE, 0>(lo, hi, v, q, g);
        if constexpr (Cfg::TM) {
            tm::wait_st();
#pragma unroll
            for (int c = 0; c < E / 16; ++c) {
                uint32_t hw[16], lw[16], zh[16], zl[16];
                tm::ld16x4(tcol + 16 * c, hw, tcol + E + 16 * c, lw, tcol + 2 * E + 16 * c, zh,
                           tcol + 3 * E + 16 * c, zl);
#pragma unroll
                for (int e = 0; e < 16; e += 2) {
                    float2 yh, yl;
                    to_ff2(v[16 * c + e], v[16 * c + e + 1], 0x1p10f, 0x1p-11f, 0x1p-32f, yh, yl);
                    float2 za = make_float2(__uint_as_float(zh[e]), __uint_as_float(zh[e + 1]));
                    float2 zb = make_float2(__uint_as_float(zl[e]), __uint_as_float(zl[e + 1]));
                    ff_mac2(make_float2(__uint_as_float(hw[e]), __uint_as_float(hw[e + 1])),
                            make_float2(__uint_as_float(lw[e]), __uint_as_float(lw[e + 1])), yh, yl,
                            za, zb);
                    zh[e] = __float_as_uint(za.x);
                    zh[e + 1] = __float_as_uint(za.y);
                    zl[e] = __float_as_uint(zb.x);
                    zl[e + 1] = __float_as_uint(zb.y);
                }
                tm::st16(tcol + 2 * E + 16 * c, zh);
                tm::st16(tcol + 3 * E + 16 * c, zl);
            }
            tm::wait_st();
        } else {
#pragma unroll
            for (int j = 0; j < E; ++j) {
                float yh, yl;
                to_ff(v[j], -32, yh, yl);
                ff_mac(xr[j], xr[E + j], yh, yl, zr[j], zr[E + j]);
            }
        }
        if constexpr (S::NR < 2) group_sync<P>(g);
    }

    // the block's Z = (zh + zl) 2^S_ref in FP64
    double zd[E];
    if constexpr (Cfg::TM) {
#pragma unroll
        for (int c = 0; c < E / 16; ++c) {
            uint32_t zh[16], zl[16];
            tm::ld16(tcol + 2 * E + 16 * c, zh);
            tm::ld16(tcol + 3 * E + 16 * c, zl);
#pragma unroll
            for (int e = 0; e < 16; ++e)
                zd[16 * c + e] = scalbn((double)__uint_as_float(zh[e]) +
                                        (double)__uint_as_float(zl[e]), sref);
        }
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j) zd[j] = scalbn((double)zr[j] + (double)zr[E + j], sref);
    }
    if constexpr (G == 1) {
#pragma unroll
        for (int j = 0; j < E; ++j) out[final_index<float, L, LE>(q, j)] = zd[j];
    } else {
        __syncthreads();
        double *acc = reinterpret_cast<double *>(smem_raw);
        for (int i = tid; i < S::N; i += kFxThreads) acc[i] = 0.0;
        __syncthreads();
        for (int gg = 0; gg < G; ++gg) {
            if (g == gg) {
#pragma unroll
                for (int j = 0; j < E; ++j) acc[final_index<float, L, LE>(q, j)] += zd[j];
            }
            __syncthreads();
        }
        for (int i = tid; i < S::N; i += kFxThreads) out[i] = acc[i];
    }
    if constexpr (Cfg::TM) {
        tm::fence_before();
        __syncthreads();
        tm::fence_after();
        if (warp == 0) tm::dealloc(s_taddr, Cfg::COLS);
    }
}

template <int L>
cudaError_t run_fx(const SketchPlan &pl, const long long *Aq, const long long *Bq, int64_t m,
                   int64_t k, int64_t p, int d, const HashParams &hp, tab_t *tabA, tab_t *tabB,
                   const int *expA, const int *expB, double *partial, cudaStream_t s) {
    using Cfg = FxCfg<L>;
    {
        const int64_t n = (int64_t)d * pl.C * (m + p);
        int64_t gt = (n + 255) / 256;
        if (gt > 152 * 32) gt = 152 * 32;
        if (gt < 1) gt = 1;
        sketch_table_kernel<float, L, Cfg::LE><<<(unsigned)gt, 256, 0, s>>>(
            hp, d, pl.L, L, pl.C, m, p, tabA, tabB);
        cudaError_t e0 = cudaGetLastError();
        if (e0 != cudaSuccess) return e0;
    }
    auto kern = sketch_fx64_kernel<L>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Cfg::SMEM);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (int64_t)pl.nchunks * d * pl.C;
    kern<<<(unsigned)blocks, Cfg::THREADS, Cfg::SMEM, s>>>(Aq, Bq, m, k, p, pl.L, pl.C, pl.chunk, d,
                                                       tabA, tabB, expA, expB, partial);
    return cudaGetLastError();
}

}  // namespace

}  // namespace cmm

namespace cmm {

int sketch_fx64_threads(int Llo) { return Llo == 14 ? FxCfg<14>::THREADS : FxCfg<13>::THREADS; }

size_t sketch_fx64_smem(int Llo) {
    switch (Llo) {
#define CASE(L) case L: return FxCfg<L>::SMEM;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10)
        CASE(11) CASE(12) CASE(13) CASE(14)
#undef CASE
    }
    return 0;
}

cudaError_t launch_sketch_fx64(const SketchPlan &pl, const long long *Aq, const long long *Bq,
                               int64_t m, int64_t k, int64_t p, int d, const HashParams &hp,
                               tab_t *tabA, tab_t *tabB, const int *expA, const int *expB,
                               double *partial, cudaStream_t s) {
    switch (pl.Llo) {
#define CASE(L) case L: return run_fx<L>(pl, Aq, Bq, m, k, p, d, hp, tabA, tabB, expA, expB, partial, s);
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10)
        CASE(11) CASE(12) CASE(13) CASE(14)
#undef CASE
    }
    return cudaErrorInvalidValue;
}

}  // namespace cmm
