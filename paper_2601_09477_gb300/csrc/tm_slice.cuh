// tm_slice.cuh -- the 2^14-point slice of the FP32 tensor-memory kernels
// (the sketch in sketch_tm.cu and the adjoint in adjoint_tm.cu): 128 threads
// with 128 values each, two register rounds of 7 butterfly bits and one
// shared-memory round trip between them; element u of the slice at word
// u + 4 (u >> 7) (round 0: thread q holds the contiguous row u = 128 q + j,
// round 1: u = q + 128 j; both bank-conflict free).  Also the tensor-memory
// moves of a thread's own lane, the fixed-point integer scatter with the
// packed tables (padded word of the bucket in bits 0-14, sign in bit 15) and
// the bucket-occupancy count that chooses its scale.
#pragma once

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

static_assert(kTmP == 128, "one TMEM lane per thread");

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

}  // namespace

}  // namespace cmm
