// adjoint_tm.cu -- the adjoint of the mean estimator (cmm_backward) for FP32
// operands and 2^14-point frequency slices, on the layout of the FP32 sketch
// kernel with tensor memory (tm_slice.cuh).
//
// The mathematics is that of adjoint.cu: with Gs_r = (1/b) H G_r,
//     dA[i][t] = s1_r(i) sum_r (H (Gs_r o H y_{r,t}))[h1_r(i)],
//     dB[t][j] = s2_r(j) sum_r (H (Gs_r o H x_{r,t}))[h2_r(j)],
// per frequency slice, the top butterfly stages folded into the gather signs
// (and the slices' contributions added when b > 2^14).  What differs is the
// blocking: one CTA of 128 threads (two per SM) runs each of the four
// transforms per (t, r) as two register rounds of 7 bits with 128 values per
// thread, instead of three rounds of 5 bits; H x_t waits in tensor memory
// while the dA half runs.  The scatters and the gathers read the packed
// tables of the sketch (padded word of the bucket, sign with the fold), so no
// hash is evaluated in the kernel, and Gs comes as an FP32 copy (the
// transforms are FP32).
#include "tm_slice.cuh"
#include "tmem_device.cuh"

namespace cmm {

namespace {

constexpr uint32_t kAtCols = 128;   // H x_t of this thread's lane

// shared memory: the slice, then the CTA's dA column (m) and dB row (p)
size_t adj_tm_smem_bytes(int64_t m, int64_t p) {
    return ((size_t)kTmStride + (size_t)m + (size_t)p) * sizeof(float);
}

__global__ void gs_to_f32_kernel(const double *__restrict__ Gs, int64_t n, float *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)Gs[i];
}

// The 2^14-point FWHT of the values a thread holds at u = q + 128 j (v[j], as
// the forward transforms leave them), written to S in natural order (word
// u + 4 (u >> 7)).  The stages are taken in the other order than in the
// forward transform: bits 7-13 first, inside the thread's registers, then one
// column-to-row exchange through S and bits 0-6 on the rows, which are stored
// as they are -- three shared-memory passes instead of five.
__device__ __forceinline__ void back_fwht_to_smem(float *S, float (&v)[kTmE], int q) {
    reg_fwht_f32<kTmE, kTmLE>(v);
#pragma unroll
    for (int j = 0; j < kTmE; ++j) S[q + 132 * j] = v[j];
    __syncthreads();
    float4 *row = reinterpret_cast<float4 *>(S + 132 * q);
#pragma unroll
    for (int c = 0; c < kTmE / 4; ++c) {
        const float4 w = row[c];
        v[4 * c] = w.x;
        v[4 * c + 1] = w.y;
        v[4 * c + 2] = w.z;
        v[4 * c + 3] = w.w;
    }
    reg_fwht_f32<kTmE, kTmLE>(v);
#pragma unroll
    for (int c = 0; c < kTmE / 4; ++c)
        row[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
}

// acc[x] += sign * S[bucket word] for the keys x = q, q + 128, ... of one table
__device__ __forceinline__ void gather_tab(const float *S, float *acc, const tab_t *__restrict__ tab,
                                           int64_t n, int q) {
    int64_t x = q;
    for (; x + 3 * kTmP < n; x += 4 * kTmP) {
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) w[e] = __ldg(tab + x + e * kTmP);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float val = S[w[e] & 0x7fffu];
            acc[x + e * kTmP] += (w[e] & 0x8000u) ? -val : val;
        }
    }
    for (; x < n; x += kTmP) {
        const uint32_t w = __ldg(tab + x);
        const float val = S[w & 0x7fffu];
        acc[x] += (w & 0x8000u) ? -val : val;
    }
}

// One CTA: slice u_hi, inner indices [t0, t1) of its block, every repetition.
// tabA / tabB: packed tables per (r, u_hi); Gs32: (1/b) H G as FP32, d x b;
// dAt (k x m) and dBt (k x p) receive the gradients (added atomically when
// several slices contribute).
__global__ void __launch_bounds__(kTmP, 2)
adjoint_tm_kernel(const float *__restrict__ At, int64_t ldat, const float *__restrict__ Bp,
                  int64_t ldbp, int64_t m, int64_t k, int64_t p, int Lfull, int C, int64_t chunk,
                  int d, const tab_t *__restrict__ tabA, const tab_t *__restrict__ tabB,
                  const float *__restrict__ Gs32, const float *__restrict__ colmax,
                  float *__restrict__ dAt, float *__restrict__ dBt, int accumulate, int vec4) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *S = reinterpret_cast<float *>(smem_raw);
    int *Si = reinterpret_cast<int *>(smem_raw);
    float *dAc = S + kTmStride;
    float *dBr = dAc + m;
    __shared__ uint32_t s_taddr;
    __shared__ int s_red[4];
    __shared__ int s_cmax[2 * CMM_MAX_D];
    const int q = threadIdx.x, warp = q >> 5;

    const uint32_t u_hi = (uint32_t)(blockIdx.x % C);
    const int64_t blk = blockIdx.x / C;
    const int64_t t0 = blk * chunk;
    const int64_t t1 = (t0 + chunk < k) ? t0 + chunk : k;
    const int64_t b = (int64_t)1 << Lfull;

    if (warp == 0) tm::alloc(&s_taddr, kAtCols);
    for (int i = q; i < kTmStride; i += kTmP) S[i] = 0.f;
    tm::fence_before();
    __syncthreads();
    tm::fence_after();
    for (int r = 0; r < d; ++r) {
        const int64_t slot = (int64_t)r * C + u_hi;
        const int ca = table_cmax(Si, tabA + slot * m, m, q, s_red);
        const int cb = table_cmax(Si, tabB + slot * p, p, q, s_red);
        if (q == 0) {
            s_cmax[r] = ca;
            s_cmax[CMM_MAX_D + r] = cb;
        }
    }
    __syncthreads();
    const uint32_t tx = s_taddr + ((uint32_t)(32 * warp) << 16);

    float v[kTmE];
    for (int64_t t = t0; t < t1; ++t) {
        if (t + 1 < t1) {   // this CTA's next rows, into the L2 (no other CTA reads them)
            const char *na = reinterpret_cast<const char *>(At + (t + 1) * ldat);
            const char *nb = reinterpret_cast<const char *>(Bp + (t + 1) * ldbp);
            for (int64_t o = (int64_t)q * 128; o < m * 4; o += (int64_t)kTmP * 128) prefetch_l2(na + o);
            for (int64_t o = (int64_t)q * 128; o < p * 4; o += (int64_t)kTmP * 128) prefetch_l2(nb + o);
        }
        for (int64_t x = q; x < m; x += kTmP) dAc[x] = 0.f;
        for (int64_t x = q; x < p; x += kTmP) dBr[x] = 0.f;
        for (int r = 0; r < d; ++r) {
            const int64_t slot = (int64_t)r * C + u_hi;
            const float *gr = Gs32 + (int64_t)r * b + (int64_t)u_hi * (1 << kTmL);
            // half 0: H x_t into tensor memory; half 1: H y_t stays in v.  The
            // halves (and below, the two gradients) share one copy of the code:
            // the unrolled transforms would not fit the instruction cache twice.
#pragma unroll 1
            for (int half = 0; half < 2; ++half) {
                float sc, inv;
                fixed_scale(__ldg(colmax + (half ? k : 0) + t), s_cmax[half * CMM_MAX_D + r], sc,
                            inv);
                const float *col = half ? Bp + t * ldbp : At + t * ldat;
                const tab_t *tab = half ? tabB + slot * p : tabA + slot * m;
                const int64_t n = half ? p : m;
                if (vec4)
                    scatter_fixed_v4<16>(Si, col, tab, n, q, sc);
                else
                    scatter_fixed<32>(Si, col, tab, n, q, sc);
                __syncthreads();
                tm_fwht(S, v, q, inv);
                if (half == 0) {
#pragma unroll
                    for (int c = 0; c < kTmE / 16; ++c) tmem_st16_nowait(tx + 16 * c, v + 16 * c);
                    __syncthreads();   // every thread's exchange of the slice done before the next scatter
                }
            }
            // grad 0: dA = H (Gs o H y) gathered at the rows' buckets;
            // grad 1: dB = H (Gs o H x) gathered at the columns' buckets
#pragma unroll 1
            for (int grad = 0; grad < 2; ++grad) {
                if (grad == 0) {
#pragma unroll
                    for (int j = 0; j < kTmE; ++j) v[j] *= __ldg(gr + q + 128 * j);
                } else {
                    tmem_wait_st();
#pragma unroll
                    for (int c = 0; c < kTmE / 16; ++c) {
                        float xs[16];
                        tmem_ld16(tx + 16 * c, xs);
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            v[16 * c + e] = xs[e] * __ldg(gr + q + 128 * (16 * c + e));
                    }
                }
                back_fwht_to_smem(S, v, q);
                __syncthreads();
                if (grad == 0)
                    gather_tab(S, dAc, tabA + slot * m, m, q);
                else
                    gather_tab(S, dBr, tabB + slot * p, p, q);
                __syncthreads();
            }
            // the slice zero again for the next scatter (pad words are never written)
            {
                float4 *row = reinterpret_cast<float4 *>(S + 132 * q);
#pragma unroll
                for (int c = 0; c < kTmE / 4; ++c) row[c] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            tm::fence_before();
            __syncthreads();
            tm::fence_after();
        }
        float *da = dAt + t * m;
        float *db = dBt + t * p;
        if (accumulate) {
            for (int64_t x = q; x < m; x += kTmP) atomicAdd(da + x, dAc[x]);
            for (int64_t x = q; x < p; x += kTmP) atomicAdd(db + x, dBr[x]);
        } else {
            for (int64_t x = q; x < m; x += kTmP) da[x] = dAc[x];
            for (int64_t x = q; x < p; x += kTmP) db[x] = dBr[x];
        }
    }
    tm::fence_before();
    __syncthreads();
    tm::fence_after();
    if (warp == 0) tm::dealloc(s_taddr, kAtCols);
}

}  // namespace

int adjoint_tm_threads() { return kTmP; }
int adjoint_tm_llo() { return kTmL; }
size_t adjoint_tm_smem(int64_t m, int64_t p) { return adj_tm_smem_bytes(m, p); }

cudaError_t launch_adjoint_tm(const AdjointPlan &pl, const float *At, const float *Bp, int64_t m,
                              int64_t k, int64_t p, int d, const HashParams &hp, const double *Gs,
                              float *Gs32, tab_t *tabA, tab_t *tabB, const float *colmax,
                              float *dAt, float *dBt, cudaStream_t s) {
    {   // the sketch's packed tables for every (r, u_hi), rows of A^T then of B
        const int64_t n = (int64_t)d * pl.C * (m + p);
        int64_t g = (n + 255) / 256;
        if (g > 152 * 32) g = 152 * 32;
        if (g < 1) g = 1;
        sketch_table_kernel<float, kTmL, kTmLE><<<(unsigned)g, 256, 0, s>>>(hp, d, pl.L, kTmL,
                                                                         pl.C, m, p, tabA, tabB);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    {
        const int64_t n = (int64_t)d << pl.L;
        int64_t g = (n + 255) / 256;
        if (g > 152 * 16) g = 152 * 16;
        gs_to_f32_kernel<<<(unsigned)g, 256, 0, s>>>(Gs, n, Gs32);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (pl.C > 1) {
        cudaError_t e = cudaMemsetAsync(dAt, 0, (size_t)k * m * sizeof(float), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(dBt, 0, (size_t)k * p * sizeof(float), s);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaFuncSetAttribute(adjoint_tm_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
    if (e != cudaSuccess) return e;
    const bool vec4 = m % 4 == 0 && p % 4 == 0 && pl.ldat % 4 == 0 && pl.ldbp % 4 == 0 &&
                      reinterpret_cast<uintptr_t>(At) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(Bp) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(tabA) % 8 == 0 &&
                      reinterpret_cast<uintptr_t>(tabB) % 8 == 0;
    adjoint_tm_kernel<<<(unsigned)((int64_t)pl.nchunks * pl.C), kTmP, pl.smem, s>>>(
        At, pl.ldat, Bp, pl.ldbp, m, k, p, pl.L, pl.C, pl.chunk, d, tabA, tabB, Gs32, colmax, dAt,
        dBt, pl.C > 1 ? 1 : 0, vec4 ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace cmm
