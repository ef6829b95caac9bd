// sketch_impl.cuh -- the fused compress -> FWHT -> multiply-accumulate kernel
// (Algorithm 1, the loop over the inner index t, with the transforms of
// Sec. 3.2), shared by the FP32 and FP64 butterfly instantiations.
//
// Work decomposition.  b = 2^L is split as b = C * N with N = 2^Llo the slice
// a CTA holds in shared memory.  Writing u = (u_hi, u_lo) and the bucket
// h1(i) = (h_hi, h_lo), the transformed sketch factorises as
//     (H x_t)[u_hi, u_lo] = (H_N f)[u_lo],
//     f[v] = sum_{i : h_lo(i) = v} s1(i) (-1)^popcount(u_hi & h_hi(i)) A[i][t],
// so the CTA owning frequency slice u_hi scatters the whole column with the
// extra sign and transforms only N values: the top L - Llo butterfly stages are
// folded into the scatter and no CTA exchanges data with another.
//
// One CTA = one (repetition r, slice u_hi, block of inner indices).  Inside it,
// G groups of P threads each take every G-th t of the block.  Per t a group
//   scatters A^T[t][:] into its zeroed shared slice (shared-memory atomics),
//   transforms it (register rounds), keeps X^ in registers,
//   scatters and transforms B[t][:] the same way, and
//   accumulates Z[u] += X^[u] * Y^[u] in registers (TZ precision).
// At the end the groups' Z are summed in FP64 and the CTA writes its FP64
// partial Z for (block, r, slice) -- the cross-block reduction is FP64.
//
// FP32 butterflies take the scatter in fixed point: shared-memory FP32 atomic
// adds are far slower than integer ones, so each column is scattered as the
// 32-bit integers round(a * 2^e), with one power of two per (CTA, column)
// such that c_max * max_i |a_i| * 2^e < 2^29 (c_max: the most elements that
// share a bucket of the CTA's slice, counted once per CTA).  The bucket sums
// are exact, independent of the order of the atomics and below 2^31; round 0
// of the transform converts them to FP32 and scales back by 2^-e.  The column
// maxima come from a separate pass (launch_rowmax).  FP64 butterflies keep
// FP64 atomics.
//
// The scatter either evaluates the hashes per element (multiply-add-shift,
// two 64-bit products) or, in the single-problem kernel, reads one packed
// 16-bit word per element from a table built once per call for the CTA's
// (r, u_hi): the padded shared-memory word of the bucket in bits 0-14 and the
// combined sign in bit 15.  The table is re-read for every t and stays in L1;
// the operand columns are streamed past L1.
#pragma once

#include "cmm_internal.h"
#include "fwht_device.cuh"

namespace cmm {

template <typename T>
__device__ __forceinline__ T neg_if(T v, uint32_t neg) { return neg ? -v : v; }

template <typename T>
__device__ __forceinline__ T ld_stream(const T *p) {
    return __ldcs(p);   // evict-first: the columns are used once per CTA
}

// scatter one column (n values, contiguous) into the group's slice, hashing
template <typename T, int L, int LE>
__device__ __forceinline__ void scatter_column(T *Sg, const T *__restrict__ col, int64_t n,
                                               uint64_t a, uint64_t c, uint64_t as, uint64_t cs,
                                               int shift, uint32_t u_hi, int q) {
    using S = FwhtShape<T, L, LE>;
    constexpr int P = S::P;
    constexpr int B = 8;
    MasWalk hw(a, c, (uint64_t)q, P), sw(as, cs, (uint64_t)q, P);   // at x = i + e P
    int64_t i = q;
    for (; i + (B - 1) * (int64_t)P < n; i += B * (int64_t)P) {
        T val[B];
#pragma unroll
        for (int e = 0; e < B; ++e) val[e] = ld_stream(col + i + e * (int64_t)P);
#pragma unroll
        for (int e = 0; e < B; ++e) {
            const uint32_t h = hw.top(shift);
            const uint32_t neg = sw.top(63) ^ (__popc((h >> L) & u_hi) & 1u);
            hw.next();
            sw.next();
            atomicAdd(Sg + pad_index<T, L, LE>((int)(h & (S::N - 1))), neg_if(val[e], neg));
        }
    }
    if (i < n) {   // the last, partial batch: all loads first
        T val[B];
#pragma unroll
        for (int e = 0; e < B; ++e)
            val[e] = i + e * (int64_t)P < n ? ld_stream(col + i + e * (int64_t)P) : T(0);
#pragma unroll
        for (int e = 0; e < B; ++e) {
            const uint32_t h = hw.top(shift);
            const uint32_t neg = sw.top(63) ^ (__popc((h >> L) & u_hi) & 1u);
            hw.next();
            sw.next();
            if (i + e * (int64_t)P < n)
                atomicAdd(Sg + pad_index<T, L, LE>((int)(h & (S::N - 1))), neg_if(val[e], neg));
        }
    }
}

// scatter one column using the packed (padded word | sign << 15) table
template <typename T, int L, int LE, int B = 8>
__device__ __forceinline__ void scatter_table(T *Sg, const T *__restrict__ col,
                                              const tab_t *__restrict__ tab, int64_t n, int q) {
    constexpr int P = FwhtShape<T, L, LE>::P;
    int64_t i = q;
    for (; i + (B - 1) * (int64_t)P < n; i += B * (int64_t)P) {
        T val[B];
        tab_t w[B];
#pragma unroll
        for (int e = 0; e < B; ++e) {
            val[e] = ld_stream(col + i + e * (int64_t)P);
            w[e] = __ldg(tab + i + e * (int64_t)P);
        }
#pragma unroll
        for (int e = 0; e < B; ++e) atomicAdd(Sg + (w[e] & 0x7fffu), neg_if(val[e], (uint32_t)(w[e] >> 15)));
    }
    if (i < n) {   // the last, partial batch: all loads first
        T val[B];
        tab_t w[B];
#pragma unroll
        for (int e = 0; e < B; ++e) {
            const bool ok = i + e * (int64_t)P < n;
            val[e] = ok ? ld_stream(col + i + e * (int64_t)P) : T(0);
            w[e] = ok ? __ldg(tab + i + e * (int64_t)P) : (tab_t)0;
        }
#pragma unroll
        for (int e = 0; e < B; ++e)
            if (i + e * (int64_t)P < n)
                atomicAdd(Sg + (w[e] & 0x7fffu), neg_if(val[e], (uint32_t)(w[e] >> 15)));
    }
}

// ---- fixed-point scatter (FP32 butterflies) ----

// the power of two 2^e of one column: cmax * colmax * 2^e < 2^29 (a bucket sum
// stays below 2^29 + cmax, so sums and differences of two fit 32 bits), with e kept
// in [-126, 126] so that 2^e and 2^-e are normal floats
__device__ __forceinline__ void fixed_scale(float colmax, int cmax, float &s, float &inv) {
    // colmax < 2^Ec (exponent field - 126; 0 and subnormals give -126) and
    // cmax < 2^Ek, so the product is below 2^(Ec + Ek)
    const int Ec = ((__float_as_int(colmax) >> 23) & 0xff) - 126;
    const int Ek = 32 - __clz(cmax);
    const int e = min(max(29 - Ec - Ek, -126), 126);
    s = __int_as_float((127 + e) << 23);
    inv = __int_as_float((127 - e) << 23);
}

// largest number of the n keys that share a bucket of the slice: counted in
// S0 (an integer view of one zeroed slice, zero again on return) by all
// THREADS threads; keys from the table when given, else hashed
template <int L, int LE, int THREADS>
__device__ __forceinline__ int block_cmax(int *S0, const tab_t *__restrict__ tab, int64_t n,
                                          uint64_t a, uint64_t c, int shift, int *red) {
    using S = FwhtShape<float, L, LE>;
    static_assert(THREADS % 32 == 0 && THREADS <= 1024, "whole warps");
    MasWalk hw(a, c, threadIdx.x, THREADS);
    for (int64_t i = threadIdx.x; i < n; i += THREADS, hw.next()) {
        const int w = tab ? (int)(__ldg(tab + i) & 0x7fffu)
                          : pad_index<float, L, LE>((int)(hw.top(shift) & (uint32_t)(S::N - 1)));
        atomicAdd(S0 + w, 1);
    }
    __syncthreads();
    int mx = 0;
    for (int i = threadIdx.x; i < S::STRIDE; i += THREADS) {
        mx = max(mx, S0[i]);
        S0[i] = 0;
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0;
#pragma unroll
    for (int w = 0; w < THREADS / 32; ++w) mx = max(mx, red[w]);
    __syncthreads();
    return mx;
}

// fixed-point scatter of one column (hashing), values round(v * s)
template <int L, int LE>
__device__ __forceinline__ void scatter_column_fixed(int *Sg, const float *__restrict__ col,
                                                     int64_t n, uint64_t a, uint64_t c,
                                                     uint64_t as, uint64_t cs, int shift,
                                                     uint32_t u_hi, int q, float s) {
    using S = FwhtShape<float, L, LE>;
    constexpr int P = S::P;
    constexpr int B = 8;
    MasWalk hw(a, c, (uint64_t)q, P), sw(as, cs, (uint64_t)q, P);   // at x = i + e P
    int64_t i = q;
    for (; i + (B - 1) * (int64_t)P < n; i += B * (int64_t)P) {
        float val[B];
#pragma unroll
        for (int e = 0; e < B; ++e) val[e] = ld_stream(col + i + e * (int64_t)P);
#pragma unroll
        for (int e = 0; e < B; ++e) {
            const uint32_t h = hw.top(shift);
            const uint32_t neg = sw.top(63) ^ (__popc((h >> L) & u_hi) & 1u);
            hw.next();
            sw.next();
            const int iv = __float2int_rn(val[e] * s);
            atomicAdd(Sg + pad_index<float, L, LE>((int)(h & (S::N - 1))), neg ? -iv : iv);
        }
    }
    if (i < n) {   // the last, partial batch: all loads first
        float val[B];
#pragma unroll
        for (int e = 0; e < B; ++e)
            val[e] = i + e * (int64_t)P < n ? ld_stream(col + i + e * (int64_t)P) : 0.f;
#pragma unroll
        for (int e = 0; e < B; ++e) {
            const uint32_t h = hw.top(shift);
            const uint32_t neg = sw.top(63) ^ (__popc((h >> L) & u_hi) & 1u);
            hw.next();
            sw.next();
            const int iv = __float2int_rn(val[e] * s);
            if (i + e * (int64_t)P < n)
                atomicAdd(Sg + pad_index<float, L, LE>((int)(h & (S::N - 1))), neg ? -iv : iv);
        }
    }
}

// fixed-point scatter of one column with the packed table, values round(v * s)
template <int L, int LE, int B = 8>
__device__ __forceinline__ void scatter_table_fixed(int *Sg, const float *__restrict__ col,
                                                    const tab_t *__restrict__ tab, int64_t n,
                                                    int q, float s) {
    constexpr int P = FwhtShape<float, L, LE>::P;
    int64_t i = q;
    for (; i + (B - 1) * (int64_t)P < n; i += B * (int64_t)P) {
        float val[B];
        tab_t w[B];
#pragma unroll
        for (int e = 0; e < B; ++e) {
            val[e] = ld_stream(col + i + e * (int64_t)P);
            w[e] = __ldg(tab + i + e * (int64_t)P);
        }
#pragma unroll
        for (int e = 0; e < B; ++e) {
            const int iv = __float2int_rn(val[e] * s);
            atomicAdd(Sg + (w[e] & 0x7fffu), (w[e] >> 15) ? -iv : iv);
        }
    }
    if (i < n) {   // the last, partial batch: all loads first
        float val[B];
        tab_t w[B];
#pragma unroll
        for (int e = 0; e < B; ++e) {
            const bool ok = i + e * (int64_t)P < n;
            val[e] = ok ? ld_stream(col + i + e * (int64_t)P) : 0.f;
            w[e] = ok ? __ldg(tab + i + e * (int64_t)P) : (tab_t)0;
        }
#pragma unroll
        for (int e = 0; e < B; ++e) {
            if (i + e * (int64_t)P < n) {
                const int iv = __float2int_rn(val[e] * s);
                atomicAdd(Sg + (w[e] & 0x7fffu), (w[e] >> 15) ? -iv : iv);
            }
        }
    }
}

// One CTA's work item: repetition r (hash functions H, or the tables tabA /
// tabB of this (r, u_hi) when not null), frequency slice u_hi, inner indices
// [t0, t1); writes its FP64 partial Z slice to `out` (N values).  cmA[t] and
// cmB[t] are the column maxima of A^T[t] and B[t] (FP32 butterflies only).
// smem_raw must hold sketch_smem_bytes<L, LE, THREADS, T>() bytes.
// L2 prefetch of the 128-byte line holding p (no fault, no result)
__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// PF: while a group works on inner index t, its threads prefetch the rows
// A^T[t + G] and B[t + G] it takes next into the L2 (for callers whose
// operands are not already there, such as the batched kernel's sketch tasks)
template <typename T, typename TZ, int L, int LE, int THREADS, bool PF = false>
__device__ __forceinline__ void sketch_block(const T *__restrict__ At, int64_t ldat,
                                             const T *__restrict__ Bp, int64_t ldbp, int64_t m,
                                             int64_t p, int Lfull, uint32_t u_hi, int64_t t0,
                                             int64_t t1, const HashRep &H,
                                             const tab_t *__restrict__ tabA,
                                             const tab_t *__restrict__ tabB,
                                             const float *__restrict__ cmA,
                                             const float *__restrict__ cmB,
                                             double *__restrict__ out, unsigned char *smem_raw) {
    using S = FwhtShape<T, L, LE>;
    constexpr int E = S::E, P = S::P, G = THREADS / P;
    constexpr bool FX = sizeof(T) == 4;   // fixed-point scatter
    static_assert(THREADS % P == 0, "CTA must hold whole groups");
    T *sm = reinterpret_cast<T *>(smem_raw);
    __shared__ int s_red[32];

    const int tid = threadIdx.x;
    const int g = tid / P, q = tid % P;
    T *Sg = sm + g * S::STRIDE;
    int *Sgi = reinterpret_cast<int *>(Sg);
    const int shift = 64 - Lfull;

    for (int i = tid; i < G * S::STRIDE; i += THREADS) sm[i] = T(0);
    __syncthreads();
    int cmaxA = 0, cmaxB = 0;
    if constexpr (FX) {
        int *S0 = reinterpret_cast<int *>(sm);
        cmaxA = block_cmax<L, LE, THREADS>(S0, tabA, m, H.a1, H.c1, shift, s_red);
        cmaxB = block_cmax<L, LE, THREADS>(S0, tabB, p, H.a2, H.c2, shift, s_red);
    }

    TZ z[E];
#pragma unroll
    for (int j = 0; j < E; ++j) z[j] = TZ(0);
    T xh[E], v[E];

    const int64_t nt = t1 > t0 ? t1 - t0 : 0;
    const int64_t iters = (nt + G - 1) / G;    // the same trip count for every group
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t t = t0 + it * G + g;
        const bool active = t < t1;
        if constexpr (PF) {
            if (t + G < t1) {
                const char *na = reinterpret_cast<const char *>(At + (t + G) * ldat);
                const char *nb = reinterpret_cast<const char *>(Bp + (t + G) * ldbp);
                for (int64_t o = (int64_t)q * 128; o < m * (int64_t)sizeof(T); o += (int64_t)P * 128)
                    prefetch_l2(na + o);
                for (int64_t o = (int64_t)q * 128; o < p * (int64_t)sizeof(T); o += (int64_t)P * 128)
                    prefetch_l2(nb + o);
            }
        }
        float sA = 1.f, invA = 1.f, sB = 1.f, invB = 1.f;
        if constexpr (FX) {
            if (active) {
                fixed_scale(__ldg(cmA + t), cmaxA, sA, invA);
                fixed_scale(__ldg(cmB + t), cmaxB, sB, invB);
            }
        }
        if (active) {
            if constexpr (FX) {
                if (tabA)
                    scatter_table_fixed<L, LE>(Sgi, At + t * ldat, tabA, m, q, sA);
                else
                    scatter_column_fixed<L, LE>(Sgi, At + t * ldat, m, H.a1, H.c1, H.as1, H.cs1,
                                                shift, u_hi, q, sA);
            } else if (tabA) {
                scatter_table<T, L, LE>(Sg, At + t * ldat, tabA, m, q);
            } else {
                scatter_column<T, L, LE>(Sg, At + t * ldat, m, H.a1, H.c1, H.as1, H.cs1, shift,
                                         u_hi, q);
            }
        }
        group_sync<P>(g);
        fwht_rounds<T, L, LE, 0, FX>(Sg, v, q, g, invA);
#pragma unroll
        for (int j = 0; j < E; ++j) xh[j] = v[j];
        group_sync<P>(g);
        if (active) {
            if constexpr (FX) {
                if (tabB)
                    scatter_table_fixed<L, LE>(Sgi, Bp + t * ldbp, tabB, p, q, sB);
                else
                    scatter_column_fixed<L, LE>(Sgi, Bp + t * ldbp, p, H.a2, H.c2, H.as2, H.cs2,
                                                shift, u_hi, q, sB);
            } else if (tabB) {
                scatter_table<T, L, LE>(Sg, Bp + t * ldbp, tabB, p, q);
            } else {
                scatter_column<T, L, LE>(Sg, Bp + t * ldbp, p, H.a2, H.c2, H.as2, H.cs2, shift,
                                         u_hi, q);
            }
        }
        group_sync<P>(g);
        fwht_rounds<T, L, LE, 0, FX>(Sg, v, q, g, invB);
        if constexpr (sizeof(TZ) == 4 && sizeof(T) == 4 && (E % 2) == 0) {
#pragma unroll
            for (int j = 0; j < E; j += 2) {
                const float2 acc = __ffma2_rn(make_float2(xh[j], xh[j + 1]),
                                              make_float2(v[j], v[j + 1]),
                                              make_float2(z[j], z[j + 1]));
                z[j] = acc.x;
                z[j + 1] = acc.y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < E; ++j) z[j] += (TZ)xh[j] * (TZ)v[j];
        }
        group_sync<P>(g);
    }

    if constexpr (G == 1) {
#pragma unroll
        for (int j = 0; j < E; ++j) out[final_index<T, L, LE>(q, j)] = (double)z[j];
    } else {
        // sum the groups' accumulators in FP64 through shared memory
        __syncthreads();
        double *acc = reinterpret_cast<double *>(smem_raw);
        for (int i = tid; i < S::N; i += THREADS) acc[i] = 0.0;
        __syncthreads();
        for (int gg = 0; gg < G; ++gg) {
            if (g == gg) {
#pragma unroll
                for (int j = 0; j < E; ++j) acc[final_index<T, L, LE>(q, j)] += (double)z[j];
            }
            __syncthreads();
        }
        for (int i = tid; i < S::N; i += THREADS) out[i] = acc[i];
    }
}

template <typename T, typename TZ, int L, int LE, int THREADS>
__global__ void __launch_bounds__(THREADS, (THREADS >= 512 ? 1 : 2))
sketch_kernel(const T *__restrict__ At, int64_t ldat, const T *__restrict__ Bp, int64_t ldbp,
              int64_t m, int64_t k, int64_t p, int Lfull, int C, int64_t chunk, int d,
              const __grid_constant__ HashParams hp, const tab_t *__restrict__ tabA,
              const tab_t *__restrict__ tabB, const float *__restrict__ colmax,
              double *__restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int item = blockIdx.x;
    const uint32_t u_hi = (uint32_t)(item % C);
    item /= C;
    const int r = item % d;
    const int64_t blk = item / d;
    const int64_t t0 = blk * chunk;
    const int64_t t1 = (t0 + chunk < k) ? t0 + chunk : k;
    const int64_t b = (int64_t)1 << Lfull;
    double *out = partial + (blk * d + r) * b + (int64_t)u_hi * (1 << L);
    const int64_t slot = (int64_t)r * C + u_hi;
    sketch_block<T, TZ, L, LE, THREADS>(At, ldat, Bp, ldbp, m, p, Lfull, u_hi, t0, t1, hp.rep[r],
                                        tabA ? tabA + slot * m : nullptr,
                                        tabB ? tabB + slot * p : nullptr, colmax,
                                        colmax ? colmax + k : nullptr, out, smem_raw);
}

// packed scatter words for every (r, u_hi) slot: tab[(r*C + u_hi)*n + x] =
// padded shared-memory word of h_lo(x) | (combined sign bit) << 15
template <typename T, int L, int LE>
__global__ void sketch_table_kernel(const __grid_constant__ HashParams hp, int d, int Lfull,
                                    int Llo, int C, int64_t m, int64_t p,
                                    tab_t *__restrict__ tabA, tab_t *__restrict__ tabB) {
    const int shift = 64 - Lfull;
    const int64_t nA = (int64_t)d * C * m, n = nA + (int64_t)d * C * p;
    const uint32_t lo_mask = (1u << Llo) - 1u;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const bool isA = e < nA;
        const int64_t f = isA ? e : e - nA;
        const int64_t len = isA ? m : p;
        const int64_t slot = f / len;
        const uint64_t x = (uint64_t)(f % len);
        const int r = (int)(slot / C);
        const uint32_t u_hi = (uint32_t)(slot % C);
        const HashRep &H = hp.rep[r];
        const uint32_t h = isA ? mas_hash(H.a1, H.c1, x, shift) : mas_hash(H.a2, H.c2, x, shift);
        const uint32_t sb = isA ? mas_sign_bit(H.as1, H.cs1, x) : mas_sign_bit(H.as2, H.cs2, x);
        const uint32_t neg = sb ^ (__popc((h >> Llo) & u_hi) & 1u);
        const tab_t w = (tab_t)(pad_index<T, L, LE>((int)(h & lo_mask)) | (neg << 15));
        if (isA)
            tabA[f] = w;
        else
            tabB[f] = w;
    }
}

// launch one instantiation; smem must be set up by the caller's attribute call
template <typename T, typename TZ, int L, int LE, int THREADS>
cudaError_t launch_sketch_inst(const SketchPlan &pl, const T *At, const T *Bp, int64_t m,
                               int64_t k, int64_t p, int d, const HashParams &hp,
                               const tab_t *tabA, const tab_t *tabB, const float *colmax,
                               double *partial, cudaStream_t s) {
    if (tabA) {
        const int64_t n = (int64_t)d * pl.C * (m + p);
        int64_t g = (n + 255) / 256;
        if (g > 152 * 32) g = 152 * 32;
        if (g < 1) g = 1;
        sketch_table_kernel<T, L, LE><<<(unsigned)g, 256, 0, s>>>(hp, d, pl.L, L, pl.C, m, p,
                                                              const_cast<tab_t *>(tabA),
                                                              const_cast<tab_t *>(tabB));
        cudaError_t e0 = cudaGetLastError();
        if (e0 != cudaSuccess) return e0;
    }
    auto kern = sketch_kernel<T, TZ, L, LE, THREADS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pl.smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (int64_t)pl.nchunks * d * pl.C;
    kern<<<(unsigned)blocks, THREADS, pl.smem, s>>>(At, pl.ldat, Bp, pl.ldbp, m, k, p, pl.L,
                                                    pl.C, pl.chunk, d, hp, tabA, tabB, colmax,
                                                    partial);
    return cudaGetLastError();
}

template <int L, int LE, int THREADS, typename T>
constexpr size_t sketch_smem_bytes() {
    using S = FwhtShape<T, L, LE>;
    constexpr int G = THREADS / S::P;
    size_t a = (size_t)G * S::STRIDE * sizeof(T);
    size_t red = G > 1 ? (size_t)S::N * sizeof(double) : 0;
    return a > red ? a : red;
}

}  // namespace cmm
