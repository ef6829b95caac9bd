// finish.cu -- the last step of Compress (Algorithm 1): the FP64 reduction of
// the per-block partial Z over the inner-index blocks, then the inverse
// transform R_r = (1/b) H Z_r (Sec. 3.2: H H = b I for the unnormalised H).
//
// b = 2^L is viewed as C_f x N_f (N_f = 2^min(L, 12)).  Pass A reduces the
// blocks and transforms along the C_f high index bits (column blocks of Z_r in
// shared memory); pass B transforms each row of N_f along the low bits and
// applies the exact power-of-two scale 1/b.  Every element goes through L
// butterfly stages in total, all FP64.
#include "cmm_internal.h"

namespace cmm {

namespace {

constexpr int kThreads = 256;

// pass A: Z[r][vh][c] for the CTA's column block, summed over blocks, then
// transformed along vh.  smem holds Ch x W doubles.
__global__ void __launch_bounds__(kThreads) finish_hi_kernel(const double *__restrict__ partial,
                                                             int nchunks, int d, int L, int Lf,
                                                             int W, double *__restrict__ Z) {
    extern __shared__ double sm[];
    const int64_t b = (int64_t)1 << L;
    const int Nf = 1 << Lf;
    const int Ch = 1 << (L - Lf);
    const int nblk = Nf / W;
    const int r = blockIdx.x / nblk;
    const int c0 = (blockIdx.x % nblk) * W;
    const int64_t stride_chunk = (int64_t)d * b;
    const double *src = partial + (int64_t)r * b;
    for (int e = threadIdx.x; e < Ch * W; e += kThreads) {
        const int vh = e / W, c = e % W;
        const int64_t off = (int64_t)vh * Nf + c0 + c;
        double s = 0.0;
        for (int ch = 0; ch < nchunks; ++ch) s += src[(int64_t)ch * stride_chunk + off];
        sm[e] = s;
    }
    __syncthreads();
    for (int h = 1; h < Ch; h <<= 1) {
        for (int e = threadIdx.x; e < (Ch / 2) * W; e += kThreads) {
            const int pair = e / W, c = e % W;
            const int lo = (pair / h) * 2 * h + (pair % h);
            const double a = sm[lo * W + c], bb = sm[(lo + h) * W + c];
            sm[lo * W + c] = a + bb;
            sm[(lo + h) * W + c] = a - bb;
        }
        __syncthreads();
    }
    double *dst = Z + (int64_t)r * b;
    for (int e = threadIdx.x; e < Ch * W; e += kThreads) {
        const int vh = e / W, c = e % W;
        dst[(int64_t)vh * Nf + c0 + c] = sm[e];
    }
}

// pass B: row u_hi of Z_r (N_f values), transformed along the low bits, / b
__global__ void __launch_bounds__(kThreads) finish_lo_kernel(const double *__restrict__ Z, int L,
                                                             int Lf, double *__restrict__ R) {
    extern __shared__ double sm[];
    const int64_t b = (int64_t)1 << L;
    const int Nf = 1 << Lf;
    const int Ch = 1 << (L - Lf);
    const int r = blockIdx.x / Ch;
    const int uh = blockIdx.x % Ch;
    const double *src = Z + (int64_t)r * b + (int64_t)uh * Nf;
    for (int e = threadIdx.x; e < Nf; e += kThreads) sm[e] = src[e];
    __syncthreads();
    for (int h = 1; h < Nf; h <<= 1) {
        for (int e = threadIdx.x; e < Nf / 2; e += kThreads) {
            const int lo = (e / h) * 2 * h + (e % h);
            const double a = sm[lo], bb = sm[lo + h];
            sm[lo] = a + bb;
            sm[lo + h] = a - bb;
        }
        __syncthreads();
    }
    const double inv_b = ldexp(1.0, -L);   // exact power of two
    double *dst = R + (int64_t)r * b + (int64_t)uh * Nf;
    for (int e = threadIdx.x; e < Nf; e += kThreads) dst[e] = sm[e] * inv_b;
}

}  // namespace

cudaError_t launch_finish(const double *partial, int nchunks, int d, int L, double *Z, double *R,
                          cudaStream_t s) {
    const int Lf = L < kFinishLlo ? L : kFinishLlo;
    const int Nf = 1 << Lf;
    const int Ch = 1 << (L - Lf);
    // column block width: at least 4 doubles (one 32-byte sector), at most
    // 16384 doubles (128 KiB) of shared memory in total
    int W = 16384 / Ch;
    if (W > 64) W = 64;
    if (W < 4) W = 4;
    if (W > Nf) W = Nf;
    const size_t smA = (size_t)Ch * W * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(finish_hi_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smA);
    if (e != cudaSuccess) return e;
    finish_hi_kernel<<<(unsigned)(d * (Nf / W)), kThreads, smA, s>>>(partial, nchunks, d, L, Lf,
                                                                     W, Z);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smB = (size_t)Nf * sizeof(double);
    finish_lo_kernel<<<(unsigned)(d * Ch), kThreads, smB, s>>>(Z, L, Lf, R);
    return cudaGetLastError();
}

}  // namespace cmm
