// extract.cu -- Decompress (Algorithm 1) on the GPU: for every requested
// (i, j) the d values s1_r(i) s2_r(j) R_r[h1_r(i) XOR h2_r(j)] are gathered
// and combined by the median (middle order statistic; mean of the two middle
// values for even d) or the mean; plus the thresholded heavy-hitter list.
//
// Signs and order are handled on the FP64 bit patterns with integer
// instructions (the FP64 pipe of this GPU is ~1/70 of the FP32 rate): a sign
// is an XOR of bit 63, and the median network compares the order-preserving
// integer key of each double (magnitude bits flipped for negatives).
#include <cstring>

#include "cmm_internal.h"
#include "extract_device.cuh"

namespace cmm {

namespace {

constexpr int kThreads = 256;
constexpr int kRowsPerBlock = 16;
// The heavy-hitter passes over a dense estimate count hits per (row, tile of
// kHhTile columns); the tile is the extraction kernel's column tile, so the
// counts come for free while Decompress writes C.
constexpr int kHhTile = kThreads;
static_assert(kHhTile == 256, "a warp reads a tile as 8 coalesced loads per lane");

// abs(e) >= tau, decided on the magnitude bits (see HhRange)
__device__ __forceinline__ bool hh_hit(double e, HhRange hr) {
    const unsigned long long mag =
        (unsigned long long)__double_as_longlong(e) & 0x7fffffffffffffffull;
    return mag >= hr.lo && mag <= hr.hi;
}

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

// Heavy hitters in one pass over the estimates: the CTA of extract_kernel's
// tile (kRowsPerBlock rows x kThreads columns) computes its estimates (and,
// with WC, writes them to C as extract_kernel does), keeps the hits' values in
// shared memory, reserves room for them with one atomic on a global candidate
// counter and writes them there in (row, column) order; per (row, tile) it
// records the count and the offset of its first candidate.  Candidates past
// `ccap` are dropped (the caller then writes the list by a second pass).
// Rows are i0 .. of this launch; H1 at stride ldh as in extract_kernel; the
// candidates carry row0 + the row (a row block's offset in the whole C).
template <int D, bool WC>
__global__ void __launch_bounds__(kThreads) hh_cand_kernel(
    const double *__restrict__ R, const uint32_t *__restrict__ H1, const uint32_t *__restrict__ H2,
    int d, int L, int64_t m, int64_t p, int64_t ldh, int64_t row0, int reduce, HhRange hr,
    double *__restrict__ C, int64_t ldc, int32_t *__restrict__ tcounts,
    int64_t *__restrict__ tsrc, int64_t ldt, unsigned long long *__restrict__ ncand, int64_t ccap,
    int32_t *__restrict__ CI, int32_t *__restrict__ CJ, double *__restrict__ CV) {
    __shared__ uint32_t h1s[kRowsPerBlock][CMM_MAX_D];
    __shared__ int s_cnt[kRowsPerBlock][kThreads / 32];   // hits per (row, warp), then its prefix
    __shared__ int s_row[kRowsPerBlock + 1];               // exclusive prefix over the rows, total
    __shared__ long long s_base;
    __shared__ double s_val[kRowsPerBlock][kThreads];
    const int64_t b = (int64_t)1 << L;
    const uint32_t mask = (uint32_t)(b - 1);
    const int64_t col_tiles = (p + kThreads - 1) / kThreads;
    const int64_t tile = blockIdx.x % col_tiles;
    const int64_t i0 = (blockIdx.x / col_tiles) * kRowsPerBlock;
    const int64_t j = tile * kThreads + threadIdx.x;
    const int dd = D > 0 ? D : d;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = threadIdx.x; e < kRowsPerBlock * dd; e += kThreads) {
        const int rr = e / dd, r = e % dd;
        h1s[rr][r] = (i0 + rr < m) ? H1[(int64_t)r * ldh + i0 + rr] : 0u;
    }
    __syncthreads();
    uint32_t hits = 0;
    if (j < p) {
        if constexpr (D > 0) {
            uint32_t h2v[D];
#pragma unroll
            for (int r = 0; r < D; ++r) h2v[r] = H2[(int64_t)r * p + j];
#pragma unroll 1
            for (int rr = 0; rr < kRowsPerBlock && i0 + rr < m; ++rr) {
                const double e = estimate_fixed<D>(R, b, mask, h1s[rr], h2v, reduce);
                if constexpr (WC) C[(i0 + rr) * ldc + j] = e;
                if (hh_hit(e, hr)) {
                    s_val[rr][threadIdx.x] = e;
                    hits |= 1u << rr;
                }
            }
        } else {
            long long v[CMM_MAX_D];
            for (int rr = 0; rr < kRowsPerBlock && i0 + rr < m; ++rr) {
                for (int r = 0; r < d; ++r)
                    v[r] = rep_key(R + r * b, h1s[rr][r], H2[(int64_t)r * p + j], mask);
                const double e = combine_generic(v, d, reduce);
                if constexpr (WC) C[(i0 + rr) * ldc + j] = e;
                if (hh_hit(e, hr)) {
                    s_val[rr][threadIdx.x] = e;
                    hits |= 1u << rr;
                }
            }
        }
    }
#pragma unroll
    for (int rr = 0; rr < kRowsPerBlock; ++rr) {
        const unsigned bal = __ballot_sync(0xffffffffu, (hits >> rr) & 1u);
        if (lane == 0) s_cnt[rr][warp] = __popc(bal);
    }
    __syncthreads();
    if (threadIdx.x < kRowsPerBlock) {   // one thread per row: warp prefix, row total
        const int rr = threadIdx.x;
        int run = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            const int c = s_cnt[rr][w];
            s_cnt[rr][w] = run;
            run += c;
        }
        s_row[rr] = run;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int rr = 0; rr < kRowsPerBlock; ++rr) {
            const int c = s_row[rr];
            s_row[rr] = run;
            run += c;
        }
        s_row[kRowsPerBlock] = run;
        s_base = run ? (long long)atomicAdd(ncand, (unsigned long long)run) : 0;
    }
    __syncthreads();
    const long long base = s_base;
#pragma unroll
    for (int rr = 0; rr < kRowsPerBlock; ++rr) {
        const bool hit = (hits >> rr) & 1u;
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            const long long pos = base + s_row[rr] + s_cnt[rr][warp] + __popc(bal & ((1u << lane) - 1u));
            if (pos < ccap) {
                CI[pos] = (int32_t)(row0 + i0 + rr);
                CJ[pos] = (int32_t)j;
                CV[pos] = s_val[rr][threadIdx.x];
            }
        }
    }
    if (threadIdx.x < kRowsPerBlock && i0 + threadIdx.x < m) {
        const int rr = threadIdx.x;
        tcounts[(i0 + rr) * ldt + tile] = s_row[rr + 1] - s_row[rr];
        tsrc[(i0 + rr) * ldt + tile] = base + s_row[rr];
    }
}

// after hh_rowscan_kernel (inclusive prefix of the tile counts per row, row
// totals) and the scan of the row totals: each (row, tile)'s candidates are
// copied to their place in the ordered list, one warp per (row, tile)
__global__ void __launch_bounds__(kThreads) hh_cand_copy_kernel(
    const int32_t *__restrict__ tinc, const int64_t *__restrict__ tsrc, int64_t ldt, int64_t m,
    int64_t nt, const int64_t *__restrict__ offsets, const int32_t *__restrict__ CI,
    const int32_t *__restrict__ CJ, const double *__restrict__ CV, int64_t ccap,
    int32_t *__restrict__ I, int32_t *__restrict__ J, double *__restrict__ V, int64_t capacity) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t item = w0; item < m * nt; item += nw) {
        const int64_t i = item / nt, t = item % nt;
        const int hi = tinc[i * ldt + t];
        const int lo = t > 0 ? tinc[i * ldt + t - 1] : 0;
        if (hi == lo) continue;
        const int64_t dst = offsets[i] + lo, src = tsrc[i * ldt + t];
        for (int e = lane; e < hi - lo; e += 32) {
            if (dst + e < capacity && src + e < ccap) {   // past ccap: the second pass writes it
                I[dst + e] = CI[src + e];
                J[dst + e] = CJ[src + e];
                V[dst + e] = CV[src + e];
            }
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

// exclusive scan of counts[0..n) into offsets[0..n] (offsets[n] = total); one
// CTA of 1024 threads, thread q owning the contiguous chunk q of the input:
// chunk sums, one block-wide scan of the 1024 sums, then each chunk's prefixes
__global__ void __launch_bounds__(1024) hh_scan_kernel(const int64_t *__restrict__ counts,
                                                       int64_t n, int64_t *__restrict__ offsets) {
    __shared__ int64_t wsum[32];
    const int q = threadIdx.x, lane = q & 31, warp = q >> 5;
    const int64_t chunk = (n + 1023) / 1024;
    const int64_t b0 = q * chunk < n ? q * chunk : n;
    const int64_t b1 = b0 + chunk < n ? b0 + chunk : n;
    int64_t s = 0;
    for (int64_t i = b0; i < b1; ++i) s += counts[i];
    int64_t inc = s;   // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int64_t w = wsum[lane], wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t v = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += v;
        }
        wsum[lane] = wi - w;   // exclusive prefix of the warp totals
    }
    __syncthreads();
    int64_t run = wsum[warp] + inc - s;
    for (int64_t i = b0; i < b1; ++i) {
        offsets[i] = run;
        run += counts[i];
    }
    if (q == 1023) offsets[n] = run;
}

// heavy hitters from R, second pass (when the candidates overflowed): the
// ordered compaction of each row's hits, estimates recomputed
template <int D>
__global__ void __launch_bounds__(kThreads) hh_write_kernel(
    const double *__restrict__ R, const uint32_t *__restrict__ H1, const uint32_t *__restrict__ H2,
    int d, int L, int64_t m, int64_t p, int reduce, HhRange hr,
    const int64_t *__restrict__ offsets, int32_t *__restrict__ I, int32_t *__restrict__ J,
    double *__restrict__ V, int64_t capacity) {
    __shared__ uint32_t h1s[CMM_MAX_D];
    __shared__ int wcount[kThreads / 32];
    const int64_t b = (int64_t)1 << L;
    const uint32_t mask = (uint32_t)(b - 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
        int64_t off = offsets[i];
        const int64_t end = offsets[i + 1];
        if (off == end || off >= capacity) continue;   // uniform across the CTA
        for (int r = threadIdx.x; r < d; r += kThreads) h1s[r] = H1[(int64_t)r * m + i];
        __syncthreads();
        for (int64_t j0 = 0; j0 < p && off < end; j0 += kThreads) {
            const int64_t j = j0 + threadIdx.x;
            double e = 0.0;
            bool hit = false;
            if (j < p) {
                e = estimate_at<D>(R, b, mask, h1s, H2, p, j, d, reduce);
                hit = hh_hit(e, hr);
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

// heavy hitters of a dense estimate, pass 1: hits per (row, tile), one warp
// per tile (8 coalesced loads per lane)
__global__ void __launch_bounds__(kThreads) hh_tile_count_kernel(const double *__restrict__ C,
                                                                 int64_t ldc, int64_t m, int64_t p,
                                                                 HhRange hr,
                                                                 int32_t *__restrict__ tcounts,
                                                                 int64_t ldt) {
    const int lane = threadIdx.x & 31;
    const int64_t nt = (p + kHhTile - 1) / kHhTile;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t item = w0; item < m * nt; item += nw) {
        const int64_t i = item / nt, t = item % nt;
        const double *row = C + i * ldc;
        double e[kHhTile / 32];
#pragma unroll
        for (int u = 0; u < kHhTile / 32; ++u) {
            const int64_t j = t * kHhTile + 32 * u + lane;
            e[u] = j < p ? __ldcs(row + j) : 0.0;
        }
        int cnt = 0;
#pragma unroll
        for (int u = 0; u < kHhTile / 32; ++u)
            cnt += __popc(__ballot_sync(0xffffffffu,
                                        t * kHhTile + 32 * u + lane < p && hh_hit(e[u], hr)));
        if (lane == 0) tcounts[i * ldt + t] = cnt;
    }
}

// per row: tcounts[i][.] replaced by its inclusive prefix over the tiles,
// counts[i] = the row total; one warp per row
__global__ void __launch_bounds__(kThreads) hh_rowscan_kernel(int32_t *__restrict__ tcounts,
                                                              int64_t ldt, int64_t m, int64_t nt,
                                                              int64_t *__restrict__ counts) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < m; i += nw) {
        int32_t *row = tcounts + i * ldt;
        int carry = 0;   // a row holds at most p < 2^31 hits
        for (int64_t t0 = 0; t0 < nt; t0 += 32) {
            const int64_t t = t0 + lane;
            int inc = t < nt ? row[t] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            if (t < nt) row[t] = carry + inc;
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (lane == 0) counts[i] = carry;
    }
}

// pass 2: the hits of tile t of row i in column order, from offset
// offsets[i] + (inclusive prefix of tile t - 1); one warp per (row, tile),
// tiles without hits (equal prefixes) skipped after two loads
__global__ void __launch_bounds__(kThreads) hh_tile_write_kernel(
    const double *__restrict__ C, int64_t ldc, int64_t m, int64_t p, HhRange hr,
    const int32_t *__restrict__ tinc, int64_t ldt, const int64_t *__restrict__ offsets,
    int32_t *__restrict__ I, int32_t *__restrict__ J, double *__restrict__ V, int64_t capacity) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const int64_t nt = (p + kHhTile - 1) / kHhTile;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t item = w0; item < m * nt; item += nw) {
        const int64_t i = item / nt, t = item % nt;
        const int hi = tinc[i * ldt + t];
        const int lo = t > 0 ? tinc[i * ldt + t - 1] : 0;
        if (hi == lo) continue;
        int64_t o = offsets[i] + lo;
        const int64_t end = offsets[i + 1] < capacity ? offsets[i + 1] : capacity;
        if (o >= end) continue;
        const double *row = C + i * ldc;
        double e[kHhTile / 32];
#pragma unroll
        for (int u = 0; u < kHhTile / 32; ++u) {
            const int64_t j = t * kHhTile + 32 * u + lane;
            e[u] = j < p ? __ldcs(row + j) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kHhTile / 32; ++u) {
            const int64_t j = t * kHhTile + 32 * u + lane;
            const bool hit = j < p && hh_hit(e[u], hr);
            const unsigned bal = __ballot_sync(0xffffffffu, hit);
            const int64_t pos = o + __popc(bal & below);
            if (hit && pos < end) {
                I[pos] = (int32_t)i;
                J[pos] = (int32_t)j;
                V[pos] = e[u];
            }
            o += __popc(bal);
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

HhRange hh_range(double tau) {
    HhRange hr;
    hr.hi = 0x7ff0000000000000ull;   // +inf
    if (tau != tau) {
        hr.lo = 1;
        hr.hi = 0;
    } else if (tau <= 0.0) {
        hr.lo = 0;
    } else {
        uint64_t bits;
        std::memcpy(&bits, &tau, sizeof bits);
        hr.lo = bits;
    }
    return hr;
}

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

int64_t hh_tiles(int64_t p) { return (p + kHhTile - 1) / kHhTile; }

cudaError_t launch_hh_tile_count(const double *C, int64_t ldc, int64_t m, int64_t p, HhRange hr,
                                 int32_t *tcounts, int64_t ldt, cudaStream_t s) {
    const int64_t items = m * hh_tiles(p);
    const unsigned g = clamp_grid((items + kThreads / 32 - 1) / (kThreads / 32));
    hh_tile_count_kernel<<<g, kThreads, 0, s>>>(C, ldc, m, p, hr, tcounts, ldt);
    return cudaGetLastError();
}

cudaError_t launch_hh_rowscan(int32_t *tcounts, int64_t ldt, int64_t m, int64_t p,
                              int64_t *counts, cudaStream_t s) {
    const unsigned g = clamp_grid((m + kThreads / 32 - 1) / (kThreads / 32));
    hh_rowscan_kernel<<<g, kThreads, 0, s>>>(tcounts, ldt, m, hh_tiles(p), counts);
    return cudaGetLastError();
}

cudaError_t launch_hh_tile_write(const double *C, int64_t ldc, int64_t m, int64_t p, HhRange hr,
                                 const int32_t *tinc, int64_t ldt, const int64_t *offsets,
                                 int32_t *I, int32_t *J, double *V, int64_t capacity,
                                 cudaStream_t s) {
    const int64_t items = m * hh_tiles(p);
    const unsigned g = clamp_grid((items + kThreads / 32 - 1) / (kThreads / 32));
    hh_tile_write_kernel<<<g, kThreads, 0, s>>>(C, ldc, m, p, hr, tinc, ldt, offsets, I, J, V,
                                                capacity);
    return cudaGetLastError();
}

template <bool WC>
cudaError_t launch_hh_cand_t(const double *R, const uint32_t *H1, const uint32_t *H2, int d, int L,
                             int64_t m, int64_t p, int64_t ldh, int64_t row0, int reduce,
                             HhRange hr, double *C, int64_t ldc, int32_t *tcounts, int64_t *tsrc,
                             int64_t ldt, unsigned long long *ncand, int64_t ccap, int32_t *CI,
                             int32_t *CJ, double *CV, cudaStream_t s) {
    const int64_t blocks = ((m + kRowsPerBlock - 1) / kRowsPerBlock) * ((p + kThreads - 1) / kThreads);
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    const unsigned g = (unsigned)blocks;
    switch (d) {
#define X(D) case D: hh_cand_kernel<D, WC><<<g, kThreads, 0, s>>>(R, H1, H2, d, L, m, p, ldh, row0, reduce, hr, C, ldc, tcounts, tsrc, ldt, ncand, ccap, CI, CJ, CV); break;
        CMM_ODD_D_CASES(X)
#undef X
        default: hh_cand_kernel<0, WC><<<g, kThreads, 0, s>>>(R, H1, H2, d, L, m, p, ldh, row0, reduce, hr, C, ldc, tcounts, tsrc, ldt, ncand, ccap, CI, CJ, CV);
    }
    return cudaGetLastError();
}

cudaError_t launch_hh_cand(const double *R, const uint32_t *H1, const uint32_t *H2, int d, int L,
                           int64_t m, int64_t p, int64_t ldh, int64_t row0, int reduce, HhRange hr,
                           double *C, int64_t ldc, int32_t *tcounts, int64_t *tsrc, int64_t ldt,
                           unsigned long long *ncand, int64_t ccap, int32_t *CI, int32_t *CJ,
                           double *CV, cudaStream_t s) {
    return C ? launch_hh_cand_t<true>(R, H1, H2, d, L, m, p, ldh, row0, reduce, hr, C, ldc,
                                      tcounts, tsrc, ldt, ncand, ccap, CI, CJ, CV, s)
             : launch_hh_cand_t<false>(R, H1, H2, d, L, m, p, ldh, row0, reduce, hr, C, ldc,
                                       tcounts, tsrc, ldt, ncand, ccap, CI, CJ, CV, s);
}

cudaError_t launch_hh_cand_copy(const int32_t *tinc, const int64_t *tsrc, int64_t ldt, int64_t m,
                                int64_t p, const int64_t *offsets, const int32_t *CI,
                                const int32_t *CJ, const double *CV, int64_t ccap, int32_t *I,
                                int32_t *J, double *V, int64_t capacity, cudaStream_t s) {
    const int64_t items = m * hh_tiles(p);
    const unsigned g = clamp_grid((items + kThreads / 32 - 1) / (kThreads / 32));
    hh_cand_copy_kernel<<<g, kThreads, 0, s>>>(tinc, tsrc, ldt, m, hh_tiles(p), offsets, CI, CJ,
                                               CV, ccap, I, J, V, capacity);
    return cudaGetLastError();
}

cudaError_t launch_hh_scan(int64_t *counts, int64_t ntiles, cudaStream_t s) {
    // counts has 2*ntiles+1 slots: [0, ntiles) the counts, [ntiles, 2 ntiles] the offsets
    hh_scan_kernel<<<1, 1024, 0, s>>>(counts, ntiles, counts + ntiles);
    return cudaGetLastError();
}

cudaError_t launch_hh_write(const double *R, const uint32_t *H1, const uint32_t *H2, int d, int L,
                            int64_t m, int64_t p, int reduce, HhRange hr, const int64_t *offsets,
                            int32_t *I, int32_t *J, double *V, int64_t capacity, cudaStream_t s) {
    const unsigned g = clamp_grid(m);
    switch (d) {
#define X(D) case D: hh_write_kernel<D><<<g, kThreads, 0, s>>>(R, H1, H2, d, L, m, p, reduce, hr, offsets, I, J, V, capacity); break;
        CMM_ODD_D_CASES(X)
#undef X
        default: hh_write_kernel<0><<<g, kThreads, 0, s>>>(R, H1, H2, d, L, m, p, reduce, hr, offsets, I, J, V, capacity);
    }
    return cudaGetLastError();
}

cudaError_t launch_mean_pairs(const double *R, const HashParams &hp, int d, int L, int64_t P,
                              const int32_t *I, const int32_t *J, double *out, cudaStream_t s) {
    mean_pairs_kernel<<<clamp_grid((P + 255) / 256), 256, 0, s>>>(R, hp, d, L, P, I, J, out);
    return cudaGetLastError();
}

}  // namespace cmm
