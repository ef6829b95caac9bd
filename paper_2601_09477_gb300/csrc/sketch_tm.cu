// sketch_tm.cu -- FP32 sketch kernel for 2^14-point slices with the
// transformed sketch and the accumulator in tensor memory (TMEM).
//
// Same work item and mathematics as sketch_kernel (Algorithm 1's loop over t,
// frequency-split FWHT, FP32 multiply-accumulate, FP64 partial per block):
// one CTA = (repetition r, frequency slice u_hi, block of inner indices).
// What differs is the register blocking.  A CTA of 128 threads transforms the
// 2^14-point slice with 128 values per thread, so the 14 butterfly stages take
// two register rounds of 7 bits (one shared-memory round trip between them,
// instead of two with 32 values per thread).  That leaves no registers for
// H x_t and for the running sum Z, so both live in TMEM: each thread owns its
// lane's 256 columns (128 for H x_t, 128 for Z) and moves them with
// tcgen05.ld / tcgen05.st.  Two CTAs fit on an SM (2 x 256 TMEM columns),
// each with its own barriers, so one CTA's scatter overlaps the other's
// butterflies.
//
// Scatter in fixed point.  Shared-memory FP32 atomic adds are far slower than
// integer ones on this GPU, so each column is scattered as 32-bit integers:
// value a becomes round(a * 2^e), with one power of two 2^e per (CTA, column)
// chosen so that c_max * max_i |a_i| * 2^e < 2^29, c_max being the largest
// number of elements that share a bucket in this CTA's table.  Every bucket
// sum is then an exact integer below 2^31 (no overflow, no dependence on the
// order of the atomics), and it is rounded once to FP32 and scaled back by
// 2^-e when the first register round reads it.  The only error beyond FP32's
// is the quantisation of each value to a multiple of 2^-e, at most
// c_max * max|a| * 2^-28; integer-valued inputs (+-1) stay exact.
//
// Layout of the slice in shared memory: element u at word u + 4 * (u >> 7).
// Round 0: thread q holds u = 128 q + j (a contiguous, 16-byte aligned row of
// 128 words, read and written as float4); round 1: u = q + 128 j (the 32
// lanes of a warp read 32 consecutive words).  Both are bank-conflict free.
#include "tm_slice.cuh"

namespace cmm {

namespace {

// shared memory: the slice plus the TMEM address word.  Registers (about 250
// per thread) hold the SM to two CTAs, matching the 2 x 256 TMEM columns; the
// rest of the unified L1 caches the scatter tables.
constexpr size_t kTmSmem = kTmStride * sizeof(float) + 32;
constexpr uint32_t kTmCols = 256;          // 128 columns H x_t + 128 columns Z per lane
static_assert(kTmStride * 4 + 32 <= (int)kTmSmem, "slice, TMEM address and reduction words must fit");

__global__ void __launch_bounds__(kTmP, 2)
sketch_tm_kernel(const float *__restrict__ At, int64_t ldat, const float *__restrict__ Bp,
                 int64_t ldbp, int64_t m, int64_t k, int64_t p, int Lfull, int C, int64_t chunk,
                 int d, const tab_t *__restrict__ tabA, const tab_t *__restrict__ tabB,
                 const float *__restrict__ colmax, double *__restrict__ partial, int vec4) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *S = reinterpret_cast<float *>(smem_raw);
    int *Si = reinterpret_cast<int *>(smem_raw);
    uint32_t *s_taddr = reinterpret_cast<uint32_t *>(smem_raw + kTmStride * sizeof(float));
    int *s_red = reinterpret_cast<int *>(smem_raw + kTmStride * sizeof(float) + 16);
    const int q = threadIdx.x;
    const int warp = q >> 5;

    int item = blockIdx.x;
    const uint32_t u_hi = (uint32_t)(item % C);
    item /= C;
    const int r = item % d;
    const int64_t blk = item / d;
    const int64_t t0 = blk * chunk;
    const int64_t t1 = (t0 + chunk < k) ? t0 + chunk : k;
    const int64_t b = (int64_t)1 << Lfull;
    const int64_t slot = (int64_t)r * C + u_hi;
    const tab_t *tA = tabA + slot * m;
    const tab_t *tB = tabB + slot * p;
    double *out = partial + (blk * d + r) * b + (int64_t)u_hi * (1 << kTmL);

    if (warp == 0) {
        asm volatile(
            "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n\t"
            "tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;"
            :
            : "r"(smem_addr(s_taddr)), "r"(kTmCols)
            : "memory");
    }
    for (int i = q; i < kTmStride; i += kTmP) S[i] = 0.f;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // this warp's lanes: 32 * warp .. 32 * warp + 31; columns [0,128) H x, [128,256) Z
    const int cmaxA = table_cmax(Si, tA, m, q, s_red);
    const int cmaxB = table_cmax(Si, tB, p, q, s_red);
    const uint32_t tx = *s_taddr + ((uint32_t)(32 * warp) << 16);
    const uint32_t tz = tx + 128;
    {
        float zero[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) zero[e] = 0.f;
#pragma unroll
        for (int c = 0; c < kTmE / 16; ++c) tmem_st16(tz + 16 * c, zero);
    }

    float v[kTmE];
    for (int64_t t = t0; t < t1; ++t) {
        // half 0: x_t = sketch of A^T[t] -> H x_t into TMEM; half 1: y_t ->
        // Z += H x_t o H y_t.  The halves share one copy of the scatter and
        // transform code (a rolled loop keeps the unrolled transform out of
        // the instruction cache twice).  A thread's column values are all
        // loaded before its atomics (the registers of v are free then).
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            float sc, inv;
            fixed_scale(__ldg(colmax + (half ? k : 0) + t), half ? cmaxB : cmaxA, sc, inv);
            const float *col = half ? Bp + t * ldbp : At + t * ldat;
            const tab_t *tab = half ? tB : tA;
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
            } else {
#pragma unroll
                for (int c = 0; c < kTmE / 16; ++c) {
                    float xs[16], zs[16];
                    tmem_ld16x2(tx + 16 * c, xs, tz + 16 * c, zs);
#pragma unroll
                    for (int e = 0; e < 16; e += 2) {
                        const float2 acc = __ffma2_rn(make_float2(xs[e], xs[e + 1]),
                                                      make_float2(v[16 * c + e], v[16 * c + e + 1]),
                                                      make_float2(zs[e], zs[e + 1]));
                        zs[e] = acc.x;
                        zs[e + 1] = acc.y;
                    }
                    tmem_st16_nowait(tz + 16 * c, zs);
                }
            }
            tmem_wait_st();
            __syncthreads();
        }
    }

#pragma unroll
    for (int c = 0; c < kTmE / 16; ++c) {
        float zs[16];
        tmem_ld16(tz + 16 * c, zs);
#pragma unroll
        for (int e = 0; e < 16; ++e) out[q + 128 * (16 * c + e)] = (double)zs[e];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :
                     : "r"(*s_taddr), "r"(kTmCols)
                     : "memory");
    }
}

}  // namespace

bool sketch_tm_supported(int prec, int Llo) { return prec == CMM_PREC_F32 && Llo == kTmL; }
int sketch_tm_threads() { return kTmP; }
size_t sketch_tm_smem() { return kTmSmem; }

cudaError_t launch_sketch_tm_tables(const SketchPlan &pl, int64_t m, int64_t p, int d,
                                    const HashParams &hp, tab_t *tabA, tab_t *tabB,
                                    cudaStream_t s) {
    const int64_t n = (int64_t)d * pl.C * (m + p);
    int64_t g = (n + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    sketch_table_kernel<float, kTmL, kTmLE><<<(unsigned)g, 256, 0, s>>>(hp, d, pl.L, kTmL, pl.C,
                                                                     m, p, tabA, tabB);
    return cudaGetLastError();
}

cudaError_t launch_sketch_tm(const SketchPlan &pl, const float *At, const float *Bp, int64_t m,
                             int64_t k, int64_t p, int d, const tab_t *tabA, const tab_t *tabB,
                             const float *colmax, double *partial, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(sketch_tm_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmSmem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (int64_t)pl.nchunks * d * pl.C;
    // vector loads need 16-byte aligned rows of whole float4s (the tables are
    // then 8-byte aligned: slot offsets are multiples of 4 words)
    const bool vec4 = m % 4 == 0 && p % 4 == 0 && pl.ldat % 4 == 0 && pl.ldbp % 4 == 0 &&
                      reinterpret_cast<uintptr_t>(At) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(Bp) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(tabA) % 8 == 0 &&
                      reinterpret_cast<uintptr_t>(tabB) % 8 == 0;
    sketch_tm_kernel<<<(unsigned)blocks, kTmP, kTmSmem, s>>>(At, pl.ldat, Bp, pl.ldbp, m, k, p,
                                                             pl.L, pl.C, pl.chunk, d, tabA, tabB,
                                                             colmax, partial, vec4 ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace cmm
