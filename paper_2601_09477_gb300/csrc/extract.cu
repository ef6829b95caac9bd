// extract.cu -- Decompress (Algorithm 1) on the GPU: for every requested
// (i, j) the d values s1_r(i) s2_r(j) R_r[h1_r(i) XOR h2_r(j)] are gathered
// and combined by the median (middle order statistic; mean of the two middle
// values for even d) or the mean; plus the thresholded heavy-hitter list.
//
// Signs and order are handled on the FP64 bit patterns with integer
// instructions (the FP64 pipe of this GPU is ~1/70 of the FP32 rate): a sign
// is an XOR of bit 63, and the median network compares the order-preserving
// integer key of each double (magnitude bits flipped for negatives).
#include "cmm_internal.h"
#include "extract_device.cuh"

namespace cmm {

namespace {

constexpr int kThreads = 256;
constexpr int kRowsPerBlock = 16;

__global__ void hash_tables_kernel(const __grid_constant__ HashParams hp, int d, int L, int64_t m,
                                   int64_t p, uint32_t *__restrict__ H1, uint32_t *__restrict__ H2) {
    const int shift = 64 - L;
    const int64_t n1 = (int64_t)d * m, n = n1 + (int64_t)d * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < n1) {
            const int r = (int)(e / m);
            const uint64_t x = (uint64_t)(e % m);
            const HashRep &h = hp.rep[r];
            const uint32_t bkt = (uint32_t)((h.a1 * x + h.c1) >> shift);
            const uint32_t sg = (uint32_t)((h.as1 * x + h.cs1) >> 63);
            H1[e] = bkt | (sg << 31);
        } else {
            const int64_t f = e - n1;
            const int r = (int)(f / p);
            const uint64_t x = (uint64_t)(f % p);
            const HashRep &h = hp.rep[r];
            const uint32_t bkt = (uint32_t)((h.a2 * x + h.c2) >> shift);
            const uint32_t sg = (uint32_t)((h.as2 * x + h.cs2) >> 63);
            H2[f] = bkt | (sg << 31);
        }
    }
}

// dense estimate: a CTA covers kRowsPerBlock rows x kThreads columns; each
// thread keeps its column's d hash words in registers
template <int D, bool CYC>
__global__ void __launch_bounds__(kThreads) extract_kernel(const double *__restrict__ R,
                                                           const uint32_t *__restrict__ H1,
                                                           const uint32_t *__restrict__ H2, int d,
                                                           int L, int64_t m, int64_t p, int reduce,
                                                           double *__restrict__ C, int64_t ldc,
                                                           int64_t ldh) {
    __shared__ uint32_t h1s[kRowsPerBlock][CMM_MAX_D];
    const int64_t b = (int64_t)1 << L;
    const uint32_t mask = (uint32_t)(b - 1);
    const int64_t col_tiles = (p + kThreads - 1) / kThreads;
    const int64_t i0 = (blockIdx.x / col_tiles) * kRowsPerBlock;
    const int64_t j = (blockIdx.x % col_tiles) * kThreads + threadIdx.x;
    const int dd = D > 0 ? D : d;
    for (int e = threadIdx.x; e < kRowsPerBlock * dd; e += kThreads) {
        const int rr = e / dd, r = e % dd;
        h1s[rr][r] = (i0 + rr < m) ? H1[(int64_t)r * ldh + i0 + rr] : 0u;
    }
    __syncthreads();
    if (j >= p) return;
    if constexpr (D > 0) {
        uint32_t h2v[D];
#pragma unroll
        for (int r = 0; r < D; ++r) h2v[r] = H2[(int64_t)r * p + j];
        for (int rr = 0; rr < kRowsPerBlock && i0 + rr < m; ++rr)
            C[(i0 + rr) * ldc + j] = estimate_fixed<D, CYC>(R, b, mask, h1s[rr], h2v, reduce);
    } else {
        long long v[CMM_MAX_D];
        for (int rr = 0; rr < kRowsPerBlock && i0 + rr < m; ++rr) {
            for (int r = 0; r < d; ++r)
                v[r] = rep_key<CYC>(R + r * b, h1s[rr][r], H2[(int64_t)r * p + j], mask);
            C[(i0 + rr) * ldc + j] = combine_generic(v, d, reduce);
        }
    }
}

// estimate of (i, j) for the heavy-hitter passes (row words in shared memory)
template <int D>
__device__ __forceinline__ double estimate_at(const double *__restrict__ R, int64_t b, uint32_t mask,
                                              const uint32_t *h1s, const uint32_t *__restrict__ H2,
                                              int64_t p, int64_t j, int d, int reduce) {
    if constexpr (D > 0) {
        uint32_t h2v[D];
#pragma unroll
        for (int r = 0; r < D; ++r) h2v[r] = H2[(int64_t)r * p + j];
        return estimate_fixed<D>(R, b, mask, h1s, h2v, reduce);
    } else {
        long long v[CMM_MAX_D];
        for (int r = 0; r < d; ++r) v[r] = rep_key(R + r * b, h1s[r], H2[(int64_t)r * p + j], mask);
        return combine_generic(v, d, reduce);
    }
}

// heavy hitters, pass 1: hits per row (from R when C is null, else from C)
template <int D>
__global__ void __launch_bounds__(kThreads) hh_count_kernel(
    const double *__restrict__ R, const uint32_t *__restrict__ H1, const uint32_t *__restrict__ H2,
    const double *__restrict__ C, int64_t ldc, int d, int L, int64_t m, int64_t p, int reduce,
    double tau, int64_t *__restrict__ counts) {
    __shared__ uint32_t h1s[CMM_MAX_D];
    __shared__ int64_t wsum[kThreads / 32];
    const int64_t b = (int64_t)1 << L;
    const uint32_t mask = (uint32_t)(b - 1);
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
        if (!C) {
            for (int r = threadIdx.x; r < d; r += kThreads) h1s[r] = H1[(int64_t)r * m + i];
            __syncthreads();
        }
        int64_t cnt = 0;
        for (int64_t j = threadIdx.x; j < p; j += kThreads) {
            const double e = C ? C[i * ldc + j] : estimate_at<D>(R, b, mask, h1s, H2, p, j, d, reduce);
            cnt += fabs(e) >= tau;
        }
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = cnt;
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t s = 0;
            for (int w = 0; w < kThreads / 32; ++w) s += wsum[w];
            counts[i] = s;
        }
        __syncthreads();
    }
}

// exclusive scan of counts[0..n) into offsets[0..n] (offsets[n] = total); one CTA
__global__ void __launch_bounds__(1024) hh_scan_kernel(const int64_t *__restrict__ counts,
                                                       int64_t n, int64_t *__restrict__ offsets) {
    __shared__ int64_t part[1024];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += 1024) {
        const int64_t idx = base + threadIdx.x;
        const int64_t v = idx < n ? counts[idx] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int64_t add = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
            __syncthreads();
            part[threadIdx.x] += add;
            __syncthreads();
        }
        if (idx < n) offsets[idx] = carry + part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += part[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) offsets[n] = carry;
}

// heavy hitters, pass 2: ordered compaction of each row's hits
template <int D>
__global__ void __launch_bounds__(kThreads) hh_write_kernel(
    const double *__restrict__ R, const uint32_t *__restrict__ H1, const uint32_t *__restrict__ H2,
    const double *__restrict__ C, int64_t ldc, int d, int L, int64_t m, int64_t p, int reduce,
    double tau, const int64_t *__restrict__ offsets, int32_t *__restrict__ I,
    int32_t *__restrict__ J, double *__restrict__ V, int64_t capacity) {
    __shared__ uint32_t h1s[CMM_MAX_D];
    __shared__ int wcount[kThreads / 32];
    const int64_t b = (int64_t)1 << L;
    const uint32_t mask = (uint32_t)(b - 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
        int64_t off = offsets[i];
        const int64_t end = offsets[i + 1];
        if (off == end || off >= capacity) continue;   // uniform across the CTA
        if (!C) {
            for (int r = threadIdx.x; r < d; r += kThreads) h1s[r] = H1[(int64_t)r * m + i];
            __syncthreads();
        }
        for (int64_t j0 = 0; j0 < p; j0 += kThreads) {
            const int64_t j = j0 + threadIdx.x;
            double e = 0.0;
            bool hit = false;
            if (j < p) {
                e = C ? C[i * ldc + j] : estimate_at<D>(R, b, mask, h1s, H2, p, j, d, reduce);
                hit = fabs(e) >= tau;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, hit);
            if (lane == 0) wcount[warp] = __popc(bal);
            __syncthreads();
            int before = 0, total = 0;
            for (int w = 0; w < kThreads / 32; ++w) {
                before += w < warp ? wcount[w] : 0;
                total += wcount[w];
            }
            if (hit) {
                const int64_t pos = off + before + __popc(bal & ((1u << lane) - 1u));
                if (pos < capacity) {
                    I[pos] = (int32_t)i;
                    J[pos] = (int32_t)j;
                    V[pos] = e;
                }
            }
            off += total;
            __syncthreads();
        }
    }
}

__global__ void mean_pairs_kernel(const double *__restrict__ R, const __grid_constant__ HashParams hp,
                                  int d, int L, int64_t P, const int32_t *__restrict__ I,
                                  const int32_t *__restrict__ J, double *__restrict__ out) {
    const int64_t b = (int64_t)1 << L;
    const int shift = 64 - L;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P;
         q += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t i = (uint64_t)I[q], j = (uint64_t)J[q];
        double s = 0.0;
        for (int r = 0; r < d; ++r) {
            const HashRep &h = hp.rep[r];
            const uint32_t w = (uint32_t)((h.a1 * i + h.c1) >> shift) ^
                               (uint32_t)((h.a2 * j + h.c2) >> shift);
            const uint64_t neg = ((h.as1 * i + h.cs1) >> 63) ^ ((h.as2 * j + h.cs2) >> 63);
            const unsigned long long bits =
                (unsigned long long)__double_as_longlong(R[r * b + w]) ^ (neg << 63);
            s += __longlong_as_double((long long)bits);
        }
        out[q] = s / d;
    }
}

unsigned clamp_grid(int64_t g) {
    if (g < 1) return 1;
    if (g > 152 * 64) return 152 * 64;
    return (unsigned)g;
}

}  // namespace

cudaError_t launch_hash_tables(const HashParams &hp, int d, int L, int64_t m, int64_t p,
                               uint32_t *H1, uint32_t *H2, cudaStream_t s) {
    const int64_t n = (int64_t)d * (m + p);
    hash_tables_kernel<<<clamp_grid((n + 255) / 256), 256, 0, s>>>(hp, d, L, m, p, H1, H2);
    return cudaGetLastError();
}

#define CMM_ODD_D_CASES(X) X(1) X(3) X(5) X(7) X(9) X(11) X(13) X(15) X(17) X(19) X(21) X(23) \
    X(25) X(27) X(29) X(31) X(33)

template <bool CYC>
cudaError_t launch_extract_t(const double *R, const uint32_t *H1, const uint32_t *H2, int d, int L,
                             int64_t m, int64_t p, int reduce, double *C, int64_t ldc, int64_t ldh,
                             cudaStream_t s) {
    const int64_t blocks = ((m + kRowsPerBlock - 1) / kRowsPerBlock) * ((p + kThreads - 1) / kThreads);
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    const unsigned g = (unsigned)blocks;
    switch (d) {
#define X(D) case D: extract_kernel<D, CYC><<<g, kThreads, 0, s>>>(R, H1, H2, d, L, m, p, reduce, C, ldc, ldh); break;
        CMM_ODD_D_CASES(X)
#undef X
        default: extract_kernel<0, CYC><<<g, kThreads, 0, s>>>(R, H1, H2, d, L, m, p, reduce, C, ldc, ldh);
    }
    return cudaGetLastError();
}

cudaError_t launch_extract(const double *R, const uint32_t *H1, const uint32_t *H2, int d, int L,
                           int64_t m, int64_t p, int reduce, double *C, int64_t ldc, int64_t ldh,
                           cudaStream_t s, int cyclic) {
    return cyclic ? launch_extract_t<true>(R, H1, H2, d, L, m, p, reduce, C, ldc, ldh, s)
                  : launch_extract_t<false>(R, H1, H2, d, L, m, p, reduce, C, ldc, ldh, s);
}

cudaError_t launch_hh_count(const double *R, const uint32_t *H1, const uint32_t *H2,
                            const double *C, int64_t ldc, int d, int L, int64_t m, int64_t p,
                            int reduce, double tau, int64_t, int64_t, int64_t *counts,
                            cudaStream_t s) {
    const unsigned g = clamp_grid(m);
    switch (C ? -1 : d) {
#define X(D) case D: hh_count_kernel<D><<<g, kThreads, 0, s>>>(R, H1, H2, C, ldc, d, L, m, p, reduce, tau, counts); break;
        CMM_ODD_D_CASES(X)
#undef X
        default: hh_count_kernel<0><<<g, kThreads, 0, s>>>(R, H1, H2, C, ldc, d, L, m, p, reduce, tau, counts);
    }
    return cudaGetLastError();
}

cudaError_t launch_hh_scan(int64_t *counts, int64_t ntiles, cudaStream_t s) {
    // counts has 2*ntiles+1 slots: [0, ntiles) the counts, [ntiles, 2 ntiles] the offsets
    hh_scan_kernel<<<1, 1024, 0, s>>>(counts, ntiles, counts + ntiles);
    return cudaGetLastError();
}

cudaError_t launch_hh_write(const double *R, const uint32_t *H1, const uint32_t *H2,
                            const double *C, int64_t ldc, int d, int L, int64_t m, int64_t p,
                            int reduce, double tau, int64_t, int64_t, const int64_t *offsets,
                            int32_t *I, int32_t *J, double *V, int64_t capacity, cudaStream_t s) {
    const unsigned g = clamp_grid(m);
    switch (C ? -1 : d) {
#define X(D) case D: hh_write_kernel<D><<<g, kThreads, 0, s>>>(R, H1, H2, C, ldc, d, L, m, p, reduce, tau, offsets, I, J, V, capacity); break;
        CMM_ODD_D_CASES(X)
#undef X
        default: hh_write_kernel<0><<<g, kThreads, 0, s>>>(R, H1, H2, C, ldc, d, L, m, p, reduce, tau, offsets, I, J, V, capacity);
    }
    return cudaGetLastError();
}

cudaError_t launch_mean_pairs(const double *R, const HashParams &hp, int d, int L, int64_t P,
                              const int32_t *I, const int32_t *J, double *out, cudaStream_t s) {
    mean_pairs_kernel<<<clamp_grid((P + 255) / 256), 256, 0, s>>>(R, hp, d, L, P, I, J, out);
    return cudaGetLastError();
}

}  // namespace cmm
