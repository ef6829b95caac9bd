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
#include "cmm_internal.h"
#include "fwht_device.cuh"
#include "sketch_impl.cuh"

namespace cmm {

namespace {

constexpr int kTmL = 14;
constexpr int kTmLE = 7;
constexpr int kTmE = 1 << kTmLE;           // values per thread
constexpr int kTmP = (1 << kTmL) / kTmE;   // threads per CTA
constexpr int kTmStride = (1 << kTmL) + 4 * ((1 << kTmL) >> kTmLE);
// shared memory: the slice plus the TMEM address word.  Registers (about 250
// per thread) hold the SM to two CTAs, matching the 2 x 256 TMEM columns; the
// rest of the unified L1 caches the scatter tables.
constexpr size_t kTmSmem = kTmStride * sizeof(float) + 32;
constexpr uint32_t kTmCols = 256;          // 128 columns H x_t + 128 columns Z per lane

static_assert(kTmP == 128, "one TMEM lane per thread");
static_assert(kTmStride * 4 + 32 <= (int)kTmSmem, "slice, TMEM address and reduction words must fit");

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tmem_ld16(uint32_t addr, float (&x)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(addr)
        : "memory");
#pragma unroll
    for (int e = 0; e < 16; ++e) x[e] = __uint_as_float(r[e]);
}

// two 16-column loads (x and z) under one wait
__device__ __forceinline__ void tmem_ld16x2(uint32_t ax, float (&x)[16], uint32_t az, float (&z)[16]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%33];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(ax), "r"(az)
        : "memory");
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        x[e] = __uint_as_float(r[e]);
        z[e] = __uint_as_float(r[16 + e]);
    }
}

// store without waiting; tmem_wait_st() before the columns are read again or
// the source registers are overwritten by a later st
__device__ __forceinline__ void tmem_st16_nowait(uint32_t addr, const float *x) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
        :
        : "r"(addr), "r"(__float_as_uint(x[0])), "r"(__float_as_uint(x[1])),
          "r"(__float_as_uint(x[2])), "r"(__float_as_uint(x[3])), "r"(__float_as_uint(x[4])),
          "r"(__float_as_uint(x[5])), "r"(__float_as_uint(x[6])), "r"(__float_as_uint(x[7])),
          "r"(__float_as_uint(x[8])), "r"(__float_as_uint(x[9])), "r"(__float_as_uint(x[10])),
          "r"(__float_as_uint(x[11])), "r"(__float_as_uint(x[12])), "r"(__float_as_uint(x[13])),
          "r"(__float_as_uint(x[14])), "r"(__float_as_uint(x[15]))
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t addr, const float *x) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n\t"
        "tcgen05.wait::st.sync.aligned;"
        :
        : "r"(addr), "r"(__float_as_uint(x[0])), "r"(__float_as_uint(x[1])),
          "r"(__float_as_uint(x[2])), "r"(__float_as_uint(x[3])), "r"(__float_as_uint(x[4])),
          "r"(__float_as_uint(x[5])), "r"(__float_as_uint(x[6])), "r"(__float_as_uint(x[7])),
          "r"(__float_as_uint(x[8])), "r"(__float_as_uint(x[9])), "r"(__float_as_uint(x[10])),
          "r"(__float_as_uint(x[11])), "r"(__float_as_uint(x[12])), "r"(__float_as_uint(x[13])),
          "r"(__float_as_uint(x[14])), "r"(__float_as_uint(x[15]))
        : "memory");
}

// the 2^14-point FWHT of the slice S in two register rounds; result in v
// with v[j] = element q + 128 j; the slice is left zeroed.  On entry S holds
// the integer bucket sums of the fixed-point scatter, scaled back by inv.
// The first butterfly stage runs on those integers (|sum| < 2^29 + c_max, so
// a + b and a - b are exact 32-bit integers), off the FP32 pipe, and each
// result is rounded once.
__device__ __forceinline__ void tm_fwht(float *S, float (&v)[kTmE], int q, float inv) {
    float4 *row = reinterpret_cast<float4 *>(S + 132 * q);
    const int4 *irow = reinterpret_cast<const int4 *>(row);
    const float2 inv2 = make_float2(inv, inv);
#pragma unroll
    for (int c = 0; c < kTmE / 4; ++c) {
        const int4 w = irow[c];
        const float2 lo = __fmul2_rn(make_float2(__int2float_rn(w.x + w.y), __int2float_rn(w.x - w.y)), inv2);
        const float2 hi = __fmul2_rn(make_float2(__int2float_rn(w.z + w.w), __int2float_rn(w.z - w.w)), inv2);
        v[4 * c] = lo.x;
        v[4 * c + 1] = lo.y;
        v[4 * c + 2] = hi.x;
        v[4 * c + 3] = hi.y;
    }
    reg_fwht_f32<kTmE, kTmLE, true>(v);
#pragma unroll
    for (int c = 0; c < kTmE / 4; ++c)
        row[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
    __syncthreads();
    // each word of this thread's column is read and zeroed for the next
    // scatter by one exchange (a warp's 32 lanes hit 32 distinct banks, and an
    // exchange costs the shared-memory pipe about what a load does, so this
    // replaces a load pass, a clearing pass and a barrier)
    int *Si = reinterpret_cast<int *>(S);
#pragma unroll
    for (int j = 0; j < kTmE; ++j) v[j] = __int_as_float(atomicExch(Si + q + 132 * j, 0));
    reg_fwht_f32<kTmE, kTmLE>(v);
}

// largest number of table entries that share a bucket (the slice Si must be
// zero on entry; it is zero again on return); all threads of the CTA
__device__ __forceinline__ int table_cmax(int *Si, const tab_t *__restrict__ tab, int64_t n,
                                          int q, int *red) {
    for (int64_t i = q; i < n; i += kTmP) atomicAdd(Si + (__ldg(tab + i) & 0x7fffu), 1);
    __syncthreads();
    int mx = 0;
    for (int i = q; i < kTmStride; i += kTmP) {
        mx = max(mx, Si[i]);
        Si[i] = 0;
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((q & 31) == 0) red[q >> 5] = mx;
    __syncthreads();
    mx = max(max(red[0], red[1]), max(red[2], red[3]));
    __syncthreads();
    return mx;
}

// one element of the fixed-point scatter: table word w (bucket word in bits
// 0-14, sign in bit 15); the sign is applied by flipping the sign bit of the
// scale, so round(v * s) is taken once and the atomic adds an integer
__device__ __forceinline__ void scatter_one(int *Si, uint32_t w, float v, uint32_t sbits) {
    const float sc = __uint_as_float(sbits ^ ((w << 16) & 0x80000000u));
    atomicAdd(Si + (w & 0x7fffu), __float2int_rn(v * sc));
}

// scatter one column as integers round(a * s) with the packed table
template <int B>
__device__ __forceinline__ void scatter_fixed(int *Si, const float *__restrict__ col,
                                              const tab_t *__restrict__ tab, int64_t n, int q,
                                              float s) {
    int64_t i = q;
    for (; i + (B - 1) * (int64_t)kTmP < n; i += B * (int64_t)kTmP) {
        float val[B];
        tab_t w[B];
#pragma unroll
        for (int e = 0; e < B; ++e) {
            val[e] = ld_stream(col + i + e * (int64_t)kTmP);
            w[e] = __ldg(tab + i + e * (int64_t)kTmP);
        }
#pragma unroll
        for (int e = 0; e < B; ++e) scatter_one(Si, w[e], val[e], __float_as_uint(s));
    }
    if (i < n) {   // the last, partial batch: all loads first
        float val[B];
        tab_t w[B];
#pragma unroll
        for (int e = 0; e < B; ++e) {
            const bool ok = i + e * (int64_t)kTmP < n;
            val[e] = ok ? ld_stream(col + i + e * (int64_t)kTmP) : 0.f;
            w[e] = ok ? __ldg(tab + i + e * (int64_t)kTmP) : (tab_t)0;
        }
#pragma unroll
        for (int e = 0; e < B; ++e)
            if (i + e * (int64_t)kTmP < n) scatter_one(Si, w[e], val[e], __float_as_uint(s));
    }
}

// vectorised variant: n % 4 == 0, col 16-byte and tab 8-byte aligned; thread
// q takes elements 4i .. 4i+3 for i = q, q + 128, ...; batches of BV float4
// with all their loads issued before the atomics
template <int BV>
__device__ __forceinline__ void scatter_fixed_v4(int *Si, const float *__restrict__ col,
                                                 const tab_t *__restrict__ tab, int64_t n, int q,
                                                 float s) {
    const float4 *c4 = reinterpret_cast<const float4 *>(col);
    const uint2 *t4 = reinterpret_cast<const uint2 *>(tab);
    const uint32_t sb = __float_as_uint(s);
    const int64_t n4 = n >> 2;
    int64_t i = q;
    for (; i + (BV - 1) * (int64_t)kTmP < n4; i += BV * (int64_t)kTmP) {
        float4 val[BV];
        uint2 w[BV];
#pragma unroll
        for (int e = 0; e < BV; ++e) {
            val[e] = __ldcs(c4 + i + e * (int64_t)kTmP);
            w[e] = __ldg(t4 + i + e * (int64_t)kTmP);
        }
#pragma unroll
        for (int e = 0; e < BV; ++e) {
            scatter_one(Si, w[e].x & 0xffffu, val[e].x, sb);
            scatter_one(Si, w[e].x >> 16, val[e].y, sb);
            scatter_one(Si, w[e].y & 0xffffu, val[e].z, sb);
            scatter_one(Si, w[e].y >> 16, val[e].w, sb);
        }
    }
    if (i < n4) {   // the last, partial batch: loads guarded, still all issued first
        float4 val[BV];
        uint2 w[BV];
#pragma unroll
        for (int e = 0; e < BV; ++e) {
            const bool ok = i + e * (int64_t)kTmP < n4;
            val[e] = ok ? __ldcs(c4 + i + e * (int64_t)kTmP) : make_float4(0.f, 0.f, 0.f, 0.f);
            w[e] = ok ? __ldg(t4 + i + e * (int64_t)kTmP) : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int e = 0; e < BV; ++e) {
            if (i + e * (int64_t)kTmP < n4) {
                scatter_one(Si, w[e].x & 0xffffu, val[e].x, sb);
                scatter_one(Si, w[e].x >> 16, val[e].y, sb);
                scatter_one(Si, w[e].y & 0xffffu, val[e].z, sb);
                scatter_one(Si, w[e].y >> 16, val[e].w, sb);
            }
        }
    }
}

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
