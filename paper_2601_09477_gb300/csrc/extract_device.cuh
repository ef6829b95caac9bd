// extract_device.cuh -- device helpers of Decompress (Algorithm 1): the signed
// gather of one repetition's value and the median / mean over repetitions,
// done on FP64 bit patterns with integer instructions (the FP64 pipe of this
// GPU runs at ~1/70 of the FP32 rate).  A sign is an XOR of bit 63; the median
// network compares the order-preserving integer key of each double (magnitude
// bits flipped for negatives).
#pragma once

#include "cmm_internal.h"

namespace cmm {

__device__ __forceinline__ long long key_of_bits(unsigned long long bits) {
    const long long b = (long long)bits;
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double val_of_key(long long k) {
    return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}

__device__ __forceinline__ void cmpx(long long &a, long long &b) {
    const long long lo = a < b ? a : b;
    const long long hi = a < b ? b : a;
    a = lo;
    b = hi;
}
__device__ __forceinline__ long long kmin(long long a, long long b) { return a < b ? a : b; }
__device__ __forceinline__ long long kmax(long long a, long long b) { return a < b ? b : a; }
__device__ __forceinline__ long long med3(long long a, long long b, long long c) {
    return kmax(kmin(a, b), kmin(kmax(a, b), c));
}

// median of D keys (D odd, compile time): partial bubble passes, or for D = 9
// the sorted-triples form med3(max of minima, med3 of medians, min of maxima)
template <int D>
__device__ __forceinline__ long long median_odd(long long (&v)[D]) {
    if constexpr (D == 1) {
        return v[0];
    } else if constexpr (D == 3) {
        return med3(v[0], v[1], v[2]);
    } else if constexpr (D == 9) {
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            cmpx(v[3 * g], v[3 * g + 1]);
            cmpx(v[3 * g + 1], v[3 * g + 2]);
            cmpx(v[3 * g], v[3 * g + 1]);
        }
        const long long lo = kmax(kmax(v[0], v[3]), v[6]);
        const long long mid = med3(v[1], v[4], v[7]);
        const long long hi = kmin(kmin(v[2], v[5]), v[8]);
        return med3(lo, mid, hi);
    } else {
        // after pass s the top s+1 positions hold the largest values in order
#pragma unroll
        for (int s = 0; s < (D + 1) / 2; ++s) {
#pragma unroll
            for (int j = 0; j + 1 < D - s; ++j) cmpx(v[j], v[j + 1]);
        }
        return v[(D - 1) / 2];
    }
}

// generic runtime-d combine (any d <= CMM_MAX_D)
__device__ inline double combine_generic(long long *v, int d, int reduce) {
    if (reduce == CMM_MEAN) {
        double s = 0.0;
        for (int r = 0; r < d; ++r) s += val_of_key(v[r]);
        return s / d;
    }
    for (int a = 1; a < d; ++a) {
        const long long key = v[a];
        int z = a - 1;
        while (z >= 0 && v[z] > key) {
            v[z + 1] = v[z];
            --z;
        }
        v[z + 1] = key;
    }
    if (d & 1) return val_of_key(v[d / 2]);
    return 0.5 * (val_of_key(v[d / 2 - 1]) + val_of_key(v[d / 2]));
}

// value of repetition r for packed hash words (bucket | sign << 31): bucket
// h1 XOR h2 (Algorithm 1), or (h1 + h2) mod b for the cyclic form of Sec. 3.1
// (buckets are below 2^24, so the sum's bit 31 is still the XOR of the signs).
// The random gathers bypass L1 (cached in L2 only): they almost never hit
// there, and not allocating lines saves L1TEX work (2% at n = 8192).
template <bool CYC = false>
__device__ __forceinline__ long long rep_key(const double *__restrict__ Rr, uint32_t h1, uint32_t h2,
                                             uint32_t mask) {
    const uint32_t x = CYC ? h1 + h2 : h1 ^ h2;
    const unsigned long long bits =
        (unsigned long long)__double_as_longlong(__ldcg(Rr + (x & mask))) ^
        ((unsigned long long)(x >> 31) << 63);
    return key_of_bits(bits);
}

// estimate for one (i, j): h1s = the d packed words of row i, h2v = of column j
template <int D, bool CYC = false>
__device__ __forceinline__ double estimate_fixed(const double *__restrict__ R, int64_t b,
                                                 uint32_t mask, const uint32_t *h1s,
                                                 const uint32_t (&h2v)[D], int reduce) {
    long long v[D];
#pragma unroll
    for (int r = 0; r < D; ++r) v[r] = rep_key<CYC>(R + r * b, h1s[r], h2v[r], mask);
    if (reduce == CMM_MEAN) {
        double s = 0.0;
#pragma unroll
        for (int r = 0; r < D; ++r) s += val_of_key(v[r]);
        return s / D;
    }
    return val_of_key(median_odd<D>(v));
}

}  // namespace cmm
