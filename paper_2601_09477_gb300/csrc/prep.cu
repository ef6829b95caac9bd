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

// out[t][i] = A[i][t]: 32 x 32 tiles through shared memory
template <typename TI, typename TO>
__global__ void __launch_bounds__(256) transpose_kernel(const TI *__restrict__ A, int64_t lda,
                                                        int64_t m, int64_t k, TO *__restrict__ out,
                                                        int64_t ldo) {
    __shared__ TO tile[32][33];
    const int64_t tiles_i = (m + 31) / 32, tiles_t = (k + 31) / 32;
    for (int64_t tl = blockIdx.x; tl < tiles_i * tiles_t; tl += gridDim.x) {
        const int64_t i0 = (tl % tiles_i) * 32, t0 = (tl / tiles_i) * 32;
        for (int rr = threadIdx.y; rr < 32; rr += 8) {
            const int64_t i = i0 + rr, t = t0 + threadIdx.x;
            if (i < m && t < k) tile[rr][threadIdx.x] = cvt<TO>(A[i * lda + t]);
        }
        __syncthreads();
        for (int rr = threadIdx.y; rr < 32; rr += 8) {
            const int64_t t = t0 + rr, i = i0 + threadIdx.x;
            if (i < m && t < k) out[t * ldo + i] = tile[threadIdx.x][rr];
        }
        __syncthreads();
    }
}

// out[r][c] = X[r][c] converted
template <typename TI, typename TO>
__global__ void __launch_bounds__(256) convert_kernel(const TI *__restrict__ X, int64_t ldx,
                                                      int64_t rows, int64_t cols,
                                                      TO *__restrict__ out, int64_t ldo) {
    const int64_t n = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / cols, c = e % cols;
        out[r * ldo + c] = cvt<TO>(X[r * ldx + c]);
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

template <typename TO>
cudaError_t prep_A_t(const void *A, int64_t lda, int transA, int dtype, int64_t m, int64_t k,
                     TO *At, int64_t ldat, cudaStream_t s) {
    if (transA) {   // the array is A^T (k x m): convert only
        const unsigned g = grid_for(m * k, 256 * 8);
        switch (dtype) {
            case CMM_F64: convert_kernel<double, TO><<<g, 256, 0, s>>>((const double *)A, lda, k, m, At, ldat); break;
            case CMM_F32: convert_kernel<float, TO><<<g, 256, 0, s>>>((const float *)A, lda, k, m, At, ldat); break;
            case CMM_BF16: convert_kernel<__nv_bfloat16, TO><<<g, 256, 0, s>>>((const __nv_bfloat16 *)A, lda, k, m, At, ldat); break;
            default: return cudaErrorInvalidValue;
        }
    } else {
        const unsigned g = grid_for(((m + 31) / 32) * ((k + 31) / 32), 1);
        const dim3 blk(32, 8);
        switch (dtype) {
            case CMM_F64: transpose_kernel<double, TO><<<g, blk, 0, s>>>((const double *)A, lda, m, k, At, ldat); break;
            case CMM_F32: transpose_kernel<float, TO><<<g, blk, 0, s>>>((const float *)A, lda, m, k, At, ldat); break;
            case CMM_BF16: transpose_kernel<__nv_bfloat16, TO><<<g, blk, 0, s>>>((const __nv_bfloat16 *)A, lda, m, k, At, ldat); break;
            default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

template <typename TO>
cudaError_t prep_B_t(const void *B, int64_t ldb, int dtype, int64_t k, int64_t p, TO *Bp,
                     int64_t ldbp, cudaStream_t s) {
    const unsigned g = grid_for(k * p, 256 * 8);
    switch (dtype) {
        case CMM_F64: convert_kernel<double, TO><<<g, 256, 0, s>>>((const double *)B, ldb, k, p, Bp, ldbp); break;
        case CMM_F32: convert_kernel<float, TO><<<g, 256, 0, s>>>((const float *)B, ldb, k, p, Bp, ldbp); break;
        case CMM_BF16: convert_kernel<__nv_bfloat16, TO><<<g, 256, 0, s>>>((const __nv_bfloat16 *)B, ldb, k, p, Bp, ldbp); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_prep_A(const void *A, int64_t lda, int transA, int dtype, int prec, int64_t m,
                          int64_t k, void *At, int64_t ldat, cudaStream_t s) {
    if (prec == CMM_PREC_F64)
        return prep_A_t<double>(A, lda, transA, dtype, m, k, (double *)At, ldat, s);
    return prep_A_t<float>(A, lda, transA, dtype, m, k, (float *)At, ldat, s);
}

cudaError_t launch_convert_out(const void *src, int src_f64, int64_t rows, int64_t cols,
                               int transpose, void *dst, int dst_dtype, int64_t ldd,
                               cudaStream_t s) {
    if (rows == 0 || cols == 0) return cudaSuccess;
    const dim3 blk(32, 8);
    const unsigned gt = grid_for(((rows + 31) / 32) * ((cols + 31) / 32), 1);
    const unsigned gc = grid_for(rows * cols, 256 * 8);
#define CMM_CONV(TI, TO)                                                                       \
    if (transpose)                                                                             \
        transpose_kernel<TI, TO><<<gt, blk, 0, s>>>((const TI *)src, cols, rows, cols, (TO *)dst, ldd); \
    else                                                                                       \
        convert_kernel<TI, TO><<<gc, 256, 0, s>>>((const TI *)src, cols, rows, cols, (TO *)dst, ldd);
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
                          void *Bp, int64_t ldbp, cudaStream_t s) {
    if (prec == CMM_PREC_F64) return prep_B_t<double>(B, ldb, dtype, k, p, (double *)Bp, ldbp, s);
    return prep_B_t<float>(B, ldb, dtype, k, p, (float *)Bp, ldbp, s);
}

}  // namespace cmm
