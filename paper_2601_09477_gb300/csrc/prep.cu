// prep.cu -- operand preparation for the sketch kernel: the sketch reads column
// t of A and row t of B as contiguous rows of the butterfly type, so a
// row-major A is transposed (the left operand is wanted transposed, Sec. 4.3)
// and other storage types are converted.  Skipped when the caller's arrays are
// already in that form.
#include <cuda_bf16.h>

#include "cmm_internal.h"

namespace cmm {

namespace {

template <typename TO, typename TI>
__device__ __forceinline__ TO cvt(TI v) { return (TO)v; }
template <>
__device__ __forceinline__ float cvt<float, double>(double v) { return __double2float_rn(v); }
template <>
__device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ double cvt<double, __nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

// float bits of a non-negative max: integer order is float order
__device__ __forceinline__ void atomic_max_nonneg(float *addr, float v) {
    if (v > 0.f) atomicMax(reinterpret_cast<int *>(addr), __float_as_int(v));
}

template <typename TO>
__device__ __forceinline__ float abs_of(TO v) { return fabsf((float)v); }
template <>
__device__ __forceinline__ float abs_of<double>(double) { return 0.f; }

// out[t][i] = A[i][t]: 64 x 64 tiles through shared memory, 256 threads, 16
// elements per thread in flight.  Tiles run with t fastest, so the CTAs on
// the GPU at one time read whole stretches of the same rows of A and write
// contiguous stretches of the rows of out.  With MAX (float output) also
// rmax[t] = max(rmax[t], max_i |out[t][i]|), rmax zeroed by the caller; per
// thread fmaxf from 0 (NaN values are skipped, as in rowmax_kernel), then one
// atomic per (tile, t).
template <typename TI, typename TO, bool MAX>
__global__ void __launch_bounds__(256) transpose_kernel(const TI *__restrict__ A, int64_t lda,
                                                        int64_t m, int64_t k, TO *__restrict__ out,
                                                        int64_t ldo, float *__restrict__ rmax) {
    __shared__ TO tile[64][65];
    __shared__ float red[8][64];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t tiles_t = (k + 63) / 64, tiles_i = (m + 63) / 64;
    for (int64_t tl = blockIdx.x; tl < tiles_i * tiles_t; tl += gridDim.x) {
        const int64_t t0 = (tl % tiles_t) * 64, i0 = (tl / tiles_t) * 64;
        TI v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int64_t i = i0 + ty + 8 * (u >> 1), t = t0 + tx + 32 * (u & 1);
            v[u] = (i < m && t < k) ? __ldcs(A + i * lda + t) : TI(0);
        }
        float mx0 = 0.f, mx1 = 0.f;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const TO y = cvt<TO>(v[u]);
            tile[ty + 8 * (u >> 1)][tx + 32 * (u & 1)] = y;
            if constexpr (MAX) {
                if (u & 1)
                    mx1 = fmaxf(mx1, abs_of<TO>(y));
                else
                    mx0 = fmaxf(mx0, abs_of<TO>(y));
            }
        }
        if constexpr (MAX) {
            red[ty][tx] = mx0;
            red[ty][tx + 32] = mx1;
        }
        __syncthreads();
        if constexpr (MAX) {
            if (ty < 2) {
                const int c = tx + 32 * ty;
                float r = red[0][c];
#pragma unroll
                for (int y = 1; y < 8; ++y) r = fmaxf(r, red[y][c]);
                if (t0 + c < k) atomic_max_nonneg(rmax + t0 + c, r);
            }
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int tt = ty + 8 * (u >> 1), ii = tx + 32 * (u & 1);
            const int64_t t = t0 + tt, i = i0 + ii;
            if (i < m && t < k) out[t * ldo + i] = tile[ii][tt];
        }
        __syncthreads();
    }
}

constexpr int kConvPer = 16;                     // elements per thread per work item
constexpr int kConvSpan = 256 * kConvPer;        // columns per work item

// out[r][c] = X[r][c] converted; a work item is (row, span of kConvSpan
// columns), each thread keeping kConvPer loads in flight.  With MAX (float
// output) also rmax[r] = max(rmax[r], max_c |out[r][c]|), one atomic per warp
// and item (rmax zeroed by the caller; NaN values skipped as in rowmax_kernel).
template <typename TI, typename TO, bool MAX>
__global__ void __launch_bounds__(256) convert_kernel(const TI *__restrict__ X, int64_t ldx,
                                                      int64_t rows, int64_t cols,
                                                      TO *__restrict__ out, int64_t ldo,
                                                      float *__restrict__ rmax) {
    const int64_t spans = (cols + kConvSpan - 1) / kConvSpan;
    for (int64_t w = blockIdx.x; w < rows * spans; w += gridDim.x) {
        const int64_t r = w / spans, c0 = (w % spans) * kConvSpan + threadIdx.x;
        const TI *x = X + r * ldx;
        TO *o = out + r * ldo;
        TI v[kConvPer];
#pragma unroll
        for (int u = 0; u < kConvPer; ++u) {
            const int64_t c = c0 + 256 * u;
            v[u] = c < cols ? __ldcs(x + c) : TI(0);
        }
        float mx = 0.f;
#pragma unroll
        for (int u = 0; u < kConvPer; ++u) {
            const int64_t c = c0 + 256 * u;
            if (c < cols) {
                const TO y = cvt<TO>(v[u]);
                o[c] = y;
                if constexpr (MAX) mx = fmaxf(mx, abs_of<TO>(y));
            }
        }
        if constexpr (MAX) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
            if ((threadIdx.x & 31) == 0) atomic_max_nonneg(rmax + r, mx);
        }
    }
}

// out[r] = max_c |X[r][c]| (0 for an empty row): one CTA of 256 threads per row
__global__ void __launch_bounds__(256) rowmax_kernel(const float *__restrict__ X, int64_t ldx,
                                                     int64_t rows, int64_t cols,
                                                     float *__restrict__ out) {
    __shared__ float red[8];
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const float *row = X + r * ldx;
        float mx = 0.f;
        for (int64_t c = threadIdx.x; c < cols; c += 256) mx = fmaxf(mx, fabsf(__ldcs(row + c)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m = red[0];
#pragma unroll
            for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w]);
            out[r] = m;
        }
        __syncthreads();
    }
}

unsigned grid_for(int64_t work, int64_t per_block) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g > 152 * 32) g = 152 * 32;
    return (unsigned)(g < 1 ? 1 : g);
}

template <typename TO, bool MAX>
cudaError_t prep_A_t(const void *A, int64_t lda, int transA, int dtype, int64_t m, int64_t k,
                     TO *At, int64_t ldat, float *rmax, cudaStream_t s) {
    if (transA) {   // the array is A^T (k x m): convert only
        const unsigned g = grid_for(k * ((m + kConvSpan - 1) / kConvSpan), 1);
        switch (dtype) {
            case CMM_F64: convert_kernel<double, TO, MAX><<<g, 256, 0, s>>>((const double *)A, lda, k, m, At, ldat, rmax); break;
            case CMM_F32: convert_kernel<float, TO, MAX><<<g, 256, 0, s>>>((const float *)A, lda, k, m, At, ldat, rmax); break;
            case CMM_BF16: convert_kernel<__nv_bfloat16, TO, MAX><<<g, 256, 0, s>>>((const __nv_bfloat16 *)A, lda, k, m, At, ldat, rmax); break;
            default: return cudaErrorInvalidValue;
        }
    } else {
        const unsigned g = grid_for(((m + 63) / 64) * ((k + 63) / 64), 1);
        const dim3 blk(32, 8);
        switch (dtype) {
            case CMM_F64: transpose_kernel<double, TO, MAX><<<g, blk, 0, s>>>((const double *)A, lda, m, k, At, ldat, rmax); break;
            case CMM_F32: transpose_kernel<float, TO, MAX><<<g, blk, 0, s>>>((const float *)A, lda, m, k, At, ldat, rmax); break;
            case CMM_BF16: transpose_kernel<__nv_bfloat16, TO, MAX><<<g, blk, 0, s>>>((const __nv_bfloat16 *)A, lda, m, k, At, ldat, rmax); break;
            default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

template <typename TO, bool MAX>
cudaError_t prep_B_t(const void *B, int64_t ldb, int dtype, int64_t k, int64_t p, TO *Bp,
                     int64_t ldbp, float *rmax, cudaStream_t s) {
    const unsigned g = grid_for(k * ((p + kConvSpan - 1) / kConvSpan), 1);
    switch (dtype) {
        case CMM_F64: convert_kernel<double, TO, MAX><<<g, 256, 0, s>>>((const double *)B, ldb, k, p, Bp, ldbp, rmax); break;
        case CMM_F32: convert_kernel<float, TO, MAX><<<g, 256, 0, s>>>((const float *)B, ldb, k, p, Bp, ldbp, rmax); break;
        case CMM_BF16: convert_kernel<__nv_bfloat16, TO, MAX><<<g, 256, 0, s>>>((const __nv_bfloat16 *)B, ldb, k, p, Bp, ldbp, rmax); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_prep_A(const void *A, int64_t lda, int transA, int dtype, int prec, int64_t m,
                          int64_t k, void *At, int64_t ldat, cudaStream_t s, float *rmax) {
    if (prec == CMM_PREC_F64 || prec == CMM_PREC_FX64)   // FP64 copies
        return prep_A_t<double, false>(A, lda, transA, dtype, m, k, (double *)At, ldat, nullptr, s);
    if (rmax) return prep_A_t<float, true>(A, lda, transA, dtype, m, k, (float *)At, ldat, rmax, s);
    return prep_A_t<float, false>(A, lda, transA, dtype, m, k, (float *)At, ldat, nullptr, s);
}

cudaError_t launch_convert_out(const void *src, int src_f64, int64_t rows, int64_t cols,
                               int transpose, void *dst, int dst_dtype, int64_t ldd,
                               cudaStream_t s) {
    if (rows == 0 || cols == 0) return cudaSuccess;
    const dim3 blk(32, 8);
    const unsigned gt = grid_for(((rows + 63) / 64) * ((cols + 63) / 64), 1);
    const unsigned gc = grid_for(rows * ((cols + kConvSpan - 1) / kConvSpan), 1);
#define CMM_CONV(TI, TO)                                                                       \
    if (transpose)                                                                             \
        transpose_kernel<TI, TO, false><<<gt, blk, 0, s>>>((const TI *)src, cols, rows, cols, (TO *)dst, ldd, nullptr); \
    else                                                                                       \
        convert_kernel<TI, TO, false><<<gc, 256, 0, s>>>((const TI *)src, cols, rows, cols, (TO *)dst, ldd, nullptr);
    if (src_f64 && dst_dtype == CMM_F64) { CMM_CONV(double, double) }
    else if (src_f64 && dst_dtype == CMM_F32) { CMM_CONV(double, float) }
    else if (!src_f64 && dst_dtype == CMM_F64) { CMM_CONV(float, double) }
    else if (!src_f64 && dst_dtype == CMM_F32) { CMM_CONV(float, float) }
    else return cudaErrorInvalidValue;
#undef CMM_CONV
    return cudaGetLastError();
}

cudaError_t launch_rowmax(const float *X, int64_t ldx, int64_t rows, int64_t cols, float *out,
                          cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    const int64_t g = rows < 152 * 16 ? rows : 152 * 16;
    rowmax_kernel<<<(unsigned)g, 256, 0, s>>>(X, ldx, rows, cols, out);
    return cudaGetLastError();
}

cudaError_t launch_prep_B(const void *B, int64_t ldb, int dtype, int prec, int64_t k, int64_t p,
                          void *Bp, int64_t ldbp, cudaStream_t s, float *rmax) {
    if (prec == CMM_PREC_F64 || prec == CMM_PREC_FX64)   // FP64 copies
        return prep_B_t<double, false>(B, ldb, dtype, k, p, (double *)Bp, ldbp, nullptr, s);
    if (rmax) return prep_B_t<float, true>(B, ldb, dtype, k, p, (float *)Bp, ldbp, rmax, s);
    return prep_B_t<float, false>(B, ldb, dtype, k, p, (float *)Bp, ldbp, nullptr, s);
}

}  // namespace cmm
