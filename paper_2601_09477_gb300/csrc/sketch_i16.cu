// sketch_i16.cu -- the sketch for ternary operands (every entry -1, 0 or +1,
// the +-1 "Lightbulb"-type inputs of Sec. 5.2), exact in integers, two
// inner indices per pass.
//
// For such inputs every bucket sum and every value of the Walsh-Hadamard
// transform of a column's sketch is an integer of magnitude at most m (the
// column's l1 norm), so with m, p < 2^15 it fits 16 bits.  Two columns t and
// t + 1 travel as one 32-bit word W = x_t + 2^16 x_{t+1}: the scatter and the
// butterflies are linear, so adding, subtracting and negating words (mod
// 2^32) transforms both columns at once, and each half is recovered exactly
// (x_t = W - 2^16 round(W / 2^16), |x_t| < 2^15).  One shared-memory atomic,
// one word of every shared-memory pass and one integer add per butterfly
// serve two inner indices.  The multiply-accumulate unpacks both halves and
// adds x_t y_t + x_{t+1} y_{t+1} into an int32 running sum Z, which is added
// into an exact int64 accumulator in the CTA's FP64 partial slot (L2
// resident) every `flush` pairs, before it can overflow (2 m p per pair);
// the slot is converted to FP64 once at the end.  R is therefore exact: the
// FP64 finish sums integers below 2^53.
//
// Work decomposition and layouts are those of the FP32 TMEM kernel: one CTA
// of 128 threads = (repetition r, frequency slice u_hi of 2^14 points, block
// of pairs); 128 packed words per thread in two register rounds of 7 index
// bits; padded slice layout u + 4 (u >> 7); the transformed words of A and
// the running sums in tensor memory (2 x 128 columns), two CTAs per SM.
#include "cmm_internal.h"
#include "fwht_device.cuh"
#include "sketch_impl.cuh"
#include "tmem_device.cuh"

namespace cmm {

namespace {

constexpr int kIL = 14;
constexpr int kILE = 7;
constexpr int kIE = 1 << kILE;                // packed words per thread
constexpr int kIP = (1 << kIL) / kIE;         // threads per CTA
constexpr int kIStride = (1 << kIL) + 4 * ((1 << kIL) >> kILE);
constexpr size_t kISmem = kIStride * sizeof(int);
constexpr uint32_t kICols = 256;              // 128 columns packed X^ + 128 columns Z per lane

static_assert(kIP == 128, "one TMEM lane per thread");

// ---------------------------------------------------------------- packing
// Wp[q][i] = X[2q][i] + 2^16 X[2q + 1][i] for q < ceil(k / 2) (the second
// half 0 past the last row); X is k x n (leading dimension ldx), FP64 or FP32;
// any entry other than -1, 0, 1 sets *bad.  The entries are classified by
// their bit patterns (integer compares: FP64 compares run at the FP64 rate).
__device__ __forceinline__ int ternary_of(double x, bool &ok) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFull;
    ok &= mag == 0ull || mag == 0x3FF0000000000000ull;
    return mag == 0ull ? 0 : ((b >> 63) ? -1 : 1);
}
__device__ __forceinline__ int ternary_of(float x, bool &ok) {
    const unsigned b = __float_as_uint(x);
    const unsigned mag = b & 0x7FFFFFFFu;
    ok &= mag == 0u || mag == 0x3F800000u;
    return mag == 0u ? 0 : ((b >> 31) ? -1 : 1);
}

template <typename TI>
__global__ void pack_pairs_kernel(const TI *__restrict__ X, int64_t ldx, int64_t k, int64_t n,
                                  int *__restrict__ Wp, int *__restrict__ bad) {
    const int64_t pairs = (k + 1) / 2;
    bool ok = true;
    for (int64_t q = blockIdx.x; q < pairs; q += gridDim.x) {
        const TI *ra = X + 2 * q * ldx;
        const TI *rb = X + (2 * q + 1) * ldx;
        const bool has_b = 2 * q + 1 < k;
        int *out = Wp + q * n;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            const int ia = ternary_of(__ldcs(ra + i), ok);
            const int ib = has_b ? ternary_of(__ldcs(rb + i), ok) : 0;
            out[i] = ia + 65536 * ib;
        }
    }
    if (!ok) atomicOr(bad, 1);
}

}  // namespace

cudaError_t launch_pack_pairs(const void *X, int x_f64, int64_t ldx, int64_t k, int64_t n,
                              int *Wp, int *bad, cudaStream_t s) {
    const int64_t pairs = (k + 1) / 2;
    if (pairs <= 0 || n <= 0) return cudaSuccess;
    const int64_t g = pairs < 152 * 16 ? pairs : 152 * 16;   // one row pair per CTA at a time
    if (x_f64)
        pack_pairs_kernel<double><<<(unsigned)g, 256, 0, s>>>((const double *)X, ldx, k, n, Wp, bad);
    else
        pack_pairs_kernel<float><<<(unsigned)g, 256, 0, s>>>((const float *)X, ldx, k, n, Wp, bad);
    return cudaGetLastError();
}

}  // namespace cmm

namespace cmm {

namespace {

// scatter one packed column pair: n words, the packed table (padded word of
// the bucket in bits 0-14, sign in bit 15); a negated word negates both halves
template <int B>
__device__ __forceinline__ void scatter_words(unsigned *S, const unsigned *__restrict__ col,
                                              const tab_t *__restrict__ tab, int64_t n, int q) {
    int64_t i = q;
    for (; i + (B - 1) * (int64_t)kIP < n; i += B * (int64_t)kIP) {
        unsigned w[B];
        tab_t t[B];
#pragma unroll
        for (int e = 0; e < B; ++e) {
            w[e] = __ldcs(col + i + e * (int64_t)kIP);
            t[e] = __ldg(tab + i + e * (int64_t)kIP);
        }
#pragma unroll
        for (int e = 0; e < B; ++e) atomicAdd(S + (t[e] & 0x7fffu), (t[e] >> 15) ? 0u - w[e] : w[e]);
    }
    if (i < n) {
        unsigned w[B];
        tab_t t[B];
#pragma unroll
        for (int e = 0; e < B; ++e) {
            const bool ok = i + e * (int64_t)kIP < n;
            w[e] = ok ? __ldcs(col + i + e * (int64_t)kIP) : 0u;
            t[e] = ok ? __ldg(tab + i + e * (int64_t)kIP) : (tab_t)0;
        }
#pragma unroll
        for (int e = 0; e < B; ++e)
            if (i + e * (int64_t)kIP < n) atomicAdd(S + (t[e] & 0x7fffu), (t[e] >> 15) ? 0u - w[e] : w[e]);
    }
}

// vectorised: n % 4 == 0, col 16-byte and tab 8-byte aligned; thread q takes
// words 4i .. 4i + 3 for i = q, q + 128, ...
template <int BV>
__device__ __forceinline__ void scatter_words_v4(unsigned *S, const unsigned *__restrict__ col,
                                                 const tab_t *__restrict__ tab, int64_t n, int q) {
    const uint4 *c4 = reinterpret_cast<const uint4 *>(col);
    const uint2 *t4 = reinterpret_cast<const uint2 *>(tab);
    const int64_t n4 = n >> 2;
    int64_t i = q;
    auto one = [&](uint32_t t, unsigned w) { atomicAdd(S + (t & 0x7fffu), (t & 0x8000u) ? 0u - w : w); };
    for (; i + (BV - 1) * (int64_t)kIP < n4; i += BV * (int64_t)kIP) {
        uint4 w[BV];
        uint2 t[BV];
#pragma unroll
        for (int e = 0; e < BV; ++e) {
            w[e] = __ldcs(c4 + i + e * (int64_t)kIP);
            t[e] = __ldg(t4 + i + e * (int64_t)kIP);
        }
#pragma unroll
        for (int e = 0; e < BV; ++e) {
            one(t[e].x & 0xffffu, w[e].x);
            one(t[e].x >> 16, w[e].y);
            one(t[e].y & 0xffffu, w[e].z);
            one(t[e].y >> 16, w[e].w);
        }
    }
    if (i < n4) {
        uint4 w[BV];
        uint2 t[BV];
#pragma unroll
        for (int e = 0; e < BV; ++e) {
            const bool ok = i + e * (int64_t)kIP < n4;
            w[e] = ok ? __ldcs(c4 + i + e * (int64_t)kIP) : make_uint4(0u, 0u, 0u, 0u);
            t[e] = ok ? __ldg(t4 + i + e * (int64_t)kIP) : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int e = 0; e < BV; ++e) {
            if (i + e * (int64_t)kIP < n4) {
                one(t[e].x & 0xffffu, w[e].x);
                one(t[e].x >> 16, w[e].y);
                one(t[e].y & 0xffffu, w[e].z);
                one(t[e].y >> 16, w[e].w);
            }
        }
    }
}

// the 2^14-point transform of the slice S (packed words) in two register
// rounds; result in v with v[j] = element q + 128 j; the slice is left zeroed
// (round 1 reads each word by an exchange with 0)
__device__ __forceinline__ void i16_fwht(unsigned *S, unsigned (&v)[kIE], int q) {
    uint4 *row = reinterpret_cast<uint4 *>(S + 132 * q);
#pragma unroll
    for (int c = 0; c < kIE / 4; ++c) {
        const uint4 w = row[c];
        v[4 * c] = w.x;
        v[4 * c + 1] = w.y;
        v[4 * c + 2] = w.z;
        v[4 * c + 3] = w.w;
    }
    reg_fwht_r4<unsigned, kIE, kILE>(v);
#pragma unroll
    for (int c = 0; c < kIE / 4; ++c) row[c] = make_uint4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kIE; ++j) v[j] = atomicExch(S + q + 132 * j, 0u);
    reg_fwht_r4<unsigned, kIE, kILE>(v);
}

// the two halves of a packed word (all arithmetic mod 2^32, unsigned):
// hi = round(W / 2^16), lo = W - 2^16 hi
__device__ __forceinline__ void unpack(unsigned w, int &lo, int &hi) {
    hi = (int)(w + 0x8000u) >> 16;
    lo = (int)(w - ((unsigned)hi << 16));
}


// One CTA: repetition r, slice u_hi, pairs [q0, q1) of the block.  Ap / Bp:
// packed pairs (npairs x m, npairs x p words); `flush`: pairs after which the
// int32 running sums are added into the int64 accumulator (2 m p flush < 2^31).
__global__ void __launch_bounds__(kIP, 2)
sketch_i16_kernel(const unsigned *__restrict__ Ap, const unsigned *__restrict__ Bp, int64_t m,
                  int64_t npairs, int64_t p, int Lfull, int C, int64_t chunk, int d,
                  const tab_t *__restrict__ tabA, const tab_t *__restrict__ tabB, int flush,
                  double *__restrict__ partial, int vec4) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t s_taddr;
    unsigned *S = reinterpret_cast<unsigned *>(smem_raw);
    const int q = threadIdx.x, warp = q >> 5;

    int item = blockIdx.x;
    const uint32_t u_hi = (uint32_t)(item % C);
    item /= C;
    const int r = item % d;
    const int64_t blk = item / d;
    const int64_t q0 = blk * chunk;
    const int64_t q1 = (q0 + chunk < npairs) ? q0 + chunk : npairs;
    const int64_t b = (int64_t)1 << Lfull;
    const int64_t slot = (int64_t)r * C + u_hi;
    const tab_t *tA = tabA + slot * m;
    const tab_t *tB = tabB + slot * p;
    double *out = partial + (blk * d + r) * b + (int64_t)u_hi * (1 << kIL);
    long long *acc = reinterpret_cast<long long *>(out);   // the same slot, as int64 until the end

    if (warp == 0) tm::alloc(&s_taddr, kICols);
    for (int i = q; i < kIStride; i += kIP) S[i] = 0u;
    tm::fence_before();
    __syncthreads();
    tm::fence_after();
    const uint32_t tx = s_taddr + ((uint32_t)(32 * warp) << 16);
    const uint32_t tz = tx + 128;
    uint32_t zero[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) zero[e] = 0u;
#pragma unroll
    for (int c = 0; c < kIE / 16; ++c) tm::st16(tz + 16 * c, zero);
    tm::wait_st();

    unsigned v[kIE];
    bool first = true;   // the accumulator has not been written yet
    int pending = 0;     // pairs in the int32 sums
    for (int64_t pp = q0; pp < q1; ++pp) {
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            const unsigned *col = half ? Bp + pp * p : Ap + pp * m;
            const tab_t *tab = half ? tB : tA;
            const int64_t n = half ? p : m;
            if (vec4)
                scatter_words_v4<8>(S, col, tab, n, q);
            else
                scatter_words<16>(S, col, tab, n, q);
            __syncthreads();
            i16_fwht(S, v, q);
            if (half == 0) {
#pragma unroll
                for (int c = 0; c < kIE / 16; ++c) {
                    uint32_t w[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) w[e] = v[16 * c + e];
                    tm::st16(tx + 16 * c, w);
                }
            } else {
#pragma unroll
                for (int c = 0; c < kIE / 16; ++c) {
                    uint32_t xs[16], zs[16];
                    tm::ld16(tx + 16 * c, xs);
                    tm::ld16(tz + 16 * c, zs);
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        int xl, xh, yl, yh;
                        unpack(xs[e], xl, xh);
                        unpack(v[16 * c + e], yl, yh);
                        zs[e] = (uint32_t)((int)zs[e] + xl * yl + xh * yh);
                    }
                    tm::st16(tz + 16 * c, zs);
                }
            }
            tm::wait_st();
            __syncthreads();
        }
        if (++pending == flush || pp + 1 == q1) {
            // int32 sums into the int64 accumulator (element q + 128 j of the slice)
#pragma unroll 1
            for (int c = 0; c < kIE / 16; ++c) {
                uint32_t zs[16];
                tm::ld16(tz + 16 * c, zs);
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    long long *a = acc + q + 128 * (16 * c + e);
                    *a = (first ? 0ll : *a) + (long long)(int)zs[e];
                }
                tm::st16(tz + 16 * c, zero);
            }
            tm::wait_st();
            first = false;
            pending = 0;
        }
    }
    // the accumulator as FP64 (exact: |Z| < 2^53), zeros for an empty block
#pragma unroll 4
    for (int j = 0; j < kIE; ++j) {
        double *o = out + q + 128 * j;
        *o = first ? 0.0 : (double)*reinterpret_cast<long long *>(o);
    }
    tm::fence_before();
    __syncthreads();
    tm::fence_after();
    if (warp == 0) tm::dealloc(s_taddr, kICols);
}

}  // namespace

}  // namespace cmm

namespace cmm {

bool sketch_i16_supported(int Llo) { return Llo == kIL; }
int sketch_i16_threads() { return kIP; }
size_t sketch_i16_smem() { return kISmem; }

cudaError_t launch_sketch_i16(const SketchPlan &pl, const unsigned *Ap, const unsigned *Bp,
                              int64_t m, int64_t npairs, int64_t p, int d, const HashParams &hp,
                              tab_t *tabA, tab_t *tabB, int flush, double *partial,
                              cudaStream_t s) {
    {
        const int64_t n = (int64_t)d * pl.C * (m + p);
        int64_t g = (n + 255) / 256;
        if (g > 152 * 32) g = 152 * 32;
        if (g < 1) g = 1;
        sketch_table_kernel<float, kIL, kILE><<<(unsigned)g, 256, 0, s>>>(hp, d, pl.L, kIL, pl.C,
                                                                       m, p, tabA, tabB);
        cudaError_t e0 = cudaGetLastError();
        if (e0 != cudaSuccess) return e0;
    }
    cudaError_t e = cudaFuncSetAttribute(sketch_i16_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kISmem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (int64_t)pl.nchunks * d * pl.C;
    const bool vec4 = m % 4 == 0 && p % 4 == 0 && reinterpret_cast<uintptr_t>(Ap) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(Bp) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(tabA) % 8 == 0 &&
                      reinterpret_cast<uintptr_t>(tabB) % 8 == 0;
    sketch_i16_kernel<<<(unsigned)blocks, kIP, kISmem, s>>>(Ap, Bp, m, npairs, p, pl.L, pl.C,
                                                           pl.chunk, d, tabA, tabB, flush, partial,
                                                           vec4 ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace cmm
