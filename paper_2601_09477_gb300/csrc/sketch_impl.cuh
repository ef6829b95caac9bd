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
#pragma once

#include "cmm_internal.h"
#include "fwht_device.cuh"

namespace cmm {

template <typename T>
__device__ __forceinline__ T neg_if(T v, uint32_t neg) { return neg ? -v : v; }

// scatter one column (n values, contiguous) into the group's slice
template <typename T, int L, int LE>
__device__ __forceinline__ void scatter_column(T *Sg, const T *__restrict__ col, int64_t n,
                                               uint64_t a, uint64_t c, uint64_t as, uint64_t cs,
                                               int shift, uint32_t u_hi, int q) {
    using S = FwhtShape<L, LE>;
    constexpr int P = S::P;
    constexpr int B = 8;
    int64_t i = q;
    for (; i + (B - 1) * (int64_t)P < n; i += B * (int64_t)P) {
        T val[B];
#pragma unroll
        for (int e = 0; e < B; ++e) val[e] = __ldg(col + i + e * (int64_t)P);
#pragma unroll
        for (int e = 0; e < B; ++e) {
            const uint64_t x = (uint64_t)(i + e * (int64_t)P);
            const uint32_t h = mas_hash(a, c, x, shift);
            const uint32_t neg = mas_sign_bit(as, cs, x) ^ (__popc((h >> L) & u_hi) & 1u);
            atomicAdd(Sg + pad_index<LE>((int)(h & (S::N - 1))), neg_if(val[e], neg));
        }
    }
    for (; i < n; i += P) {
        const T v = __ldg(col + i);
        const uint64_t x = (uint64_t)i;
        const uint32_t h = mas_hash(a, c, x, shift);
        const uint32_t neg = mas_sign_bit(as, cs, x) ^ (__popc((h >> L) & u_hi) & 1u);
        atomicAdd(Sg + pad_index<LE>((int)(h & (S::N - 1))), neg_if(v, neg));
    }
}

// One CTA's work item: repetition r (hash functions H), frequency slice u_hi,
// inner indices [t0, t1); writes its FP64 partial Z slice to `out` (N values).
// smem_raw must hold sketch_smem_bytes<L, LE, THREADS, T>() bytes.
template <typename T, typename TZ, int L, int LE, int THREADS>
__device__ __forceinline__ void sketch_block(const T *__restrict__ At, int64_t ldat,
                                             const T *__restrict__ Bp, int64_t ldbp, int64_t m,
                                             int64_t p, int Lfull, uint32_t u_hi, int64_t t0,
                                             int64_t t1, const HashRep &H,
                                             double *__restrict__ out, unsigned char *smem_raw) {
    using S = FwhtShape<L, LE>;
    constexpr int E = S::E, P = S::P, G = THREADS / P;
    static_assert(THREADS % P == 0, "CTA must hold whole groups");
    T *sm = reinterpret_cast<T *>(smem_raw);

    const int tid = threadIdx.x;
    const int g = tid / P, q = tid % P;
    T *Sg = sm + g * S::STRIDE;
    const int shift = 64 - Lfull;

    for (int i = tid; i < G * S::STRIDE; i += THREADS) sm[i] = T(0);
    __syncthreads();

    TZ z[E];
#pragma unroll
    for (int j = 0; j < E; ++j) z[j] = TZ(0);
    T xh[E], v[E];

    const int64_t nt = t1 > t0 ? t1 - t0 : 0;
    const int64_t iters = (nt + G - 1) / G;    // the same trip count for every group
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t t = t0 + it * G + g;
        const bool active = t < t1;
        if (active) scatter_column<T, L, LE>(Sg, At + t * ldat, m, H.a1, H.c1, H.as1, H.cs1,
                                             shift, u_hi, q);
        group_sync<P>(g);
        fwht_rounds<T, L, LE, 0>(Sg, v, q, g);
#pragma unroll
        for (int j = 0; j < E; ++j) xh[j] = v[j];
        group_sync<P>(g);
        if (active) scatter_column<T, L, LE>(Sg, Bp + t * ldbp, p, H.a2, H.c2, H.as2, H.cs2,
                                             shift, u_hi, q);
        group_sync<P>(g);
        fwht_rounds<T, L, LE, 0>(Sg, v, q, g);
#pragma unroll
        for (int j = 0; j < E; ++j) z[j] += (TZ)xh[j] * (TZ)v[j];
        group_sync<P>(g);
    }

    if constexpr (G == 1) {
#pragma unroll
        for (int j = 0; j < E; ++j) out[final_index<L, LE>(q, j)] = (double)z[j];
    } else {
        // sum the groups' accumulators in FP64 through shared memory
        __syncthreads();
        double *acc = reinterpret_cast<double *>(smem_raw);
        for (int i = tid; i < S::N; i += THREADS) acc[i] = 0.0;
        __syncthreads();
        for (int gg = 0; gg < G; ++gg) {
            if (g == gg) {
#pragma unroll
                for (int j = 0; j < E; ++j) acc[final_index<L, LE>(q, j)] += (double)z[j];
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
              const __grid_constant__ HashParams hp, double *__restrict__ partial) {
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
    sketch_block<T, TZ, L, LE, THREADS>(At, ldat, Bp, ldbp, m, p, Lfull, u_hi, t0, t1, hp.rep[r],
                                        out, smem_raw);
}

// launch one instantiation; smem must be set up by the caller's attribute call
template <typename T, typename TZ, int L, int LE, int THREADS>
cudaError_t launch_sketch_inst(const SketchPlan &pl, const T *At, const T *Bp, int64_t m,
                               int64_t k, int64_t p, int d, const HashParams &hp,
                               double *partial, cudaStream_t s) {
    auto kern = sketch_kernel<T, TZ, L, LE, THREADS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pl.smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (int64_t)pl.nchunks * d * pl.C;
    kern<<<(unsigned)blocks, THREADS, pl.smem, s>>>(At, pl.ldat, Bp, pl.ldbp, m, k, p, pl.L,
                                                    pl.C, pl.chunk, d, hp, partial);
    return cudaGetLastError();
}

template <int L, int LE, int THREADS, typename T>
constexpr size_t sketch_smem_bytes() {
    using S = FwhtShape<L, LE>;
    constexpr int G = THREADS / S::P;
    size_t a = (size_t)G * S::STRIDE * sizeof(T);
    size_t red = G > 1 ? (size_t)S::N * sizeof(double) : 0;
    return a > red ? a : red;
}

}  // namespace cmm
