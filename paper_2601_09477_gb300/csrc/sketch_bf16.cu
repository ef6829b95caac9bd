// sketch_bf16.cu -- the sketch with 16-bit tensor-core Hadamard blocks (BF16
// or FP16 operands).
//
// Same work item as the FP32 kernels (Algorithm 1's loop over t, frequency
// split, FP64 partial per block of t), for 2^15-point slices.  The transform
// of a slice (15 butterfly stages) runs as two passes of exact +-1 Hadamard
// blocks on the tensor cores (mma.sync m16n8k16, BF16 operands, FP32
// accumulation):
//   pass 1, bits 0-7:  a 16x16 tile X[a][b] (u = a + 16 b + 256 tau) becomes
//                      H16 X H16 -- D1 = H16 . X, then D2 = D1 . H16, where the
//                      accumulator fragments of D1 are exactly the A-operand
//                      fragments of the second product (no data movement);
//   pass 2, bits 8-14: X2[a2][n] with u = e + 2 tau' + 256 a2 + 4096 f and
//                      n = e + 2 f becomes H16 X2 (H8 (x) I2): bits 8-11 by
//                      H16, bits 12-14 by H8 while bit 0 (already transformed
//                      in pass 1) passes through the identity factor.
// H16, H8 (x) I2 hold only 0 and +-1, exact in BF16 and FP16.  The scatter is the
// fixed-point integer scatter of the FP32 kernels (per-column power-of-two
// scale, exact bucket sums); rounding happens where a value becomes a BF16
// operand: once per bucket when pass 1 reads the integer slice, the product
// inputs of pass 2, and the slice between the passes.  H x_t and the running
// sum Z stay FP32 in tensor memory (TMEM), one lane per thread.
//
// FP16 operands (template flag F16) carry 3 more significand bits than BF16
// but only 5 exponent bits, so they are scaled to a fixed range instead of
// holding real values: the integer bucket sums (|sum| < 2^30 + c_max / 2, see
// bf_scale) enter as sum * 2^-27 (< 8), the largest value that becomes an FP16
// operand is the pass-2 intermediate after 12 butterfly bits (< 2^15, below
// FP16's largest finite 65504), and each FP32 output is multiplied back by
// 2^27 and by the column scale 2^-e.  Values below 2^-14 in the scaled units
// (2^-17 of the bound) are FP16 subnormals and keep an absolute error of
// 2^-25 there.
//
// Shared memory: the integer slice (2^15 words, element u at word
// u ^ (((u >> 4) & 3) << 3): pass 1's 64-bit accesses of a half-warp hit 32
// distinct banks; pass 1 reads and clears each pair of words with one 64-bit
// exchange), then the BF16 slice between
// the passes (u at u + 2 * ((u >> 8) + 7 * (u >> 12)); pass-2 loads are
// bank-conflict free, pass-1 stores 2-way conflicted; fully rewritten by every
// pass 1, so never cleared).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cmm_internal.h"
#include "fwht_device.cuh"

namespace cmm {

namespace {

constexpr int kBL = 15;                        // log2 of the slice
constexpr int kBN = 1 << kBL;
constexpr int kBThreads = 512;                 // 16 warps
constexpr int kBWarps = kBThreads / 32;
constexpr int kBTiles = kBN / 256;             // 128 tiles of 256 per pass
constexpr int kBTilesPerWarp = kBTiles / kBWarps;   // 8
constexpr int kBElems = kBN + 2 * (127 + 7 * 7) + 2;   // padded BF16 elements
constexpr size_t kBIntBytes = (size_t)kBN * 4;          // the integer scatter slice
constexpr size_t kBBfBytes = ((size_t)kBElems * 2 + 15) / 16 * 16;
constexpr size_t kBSmem = kBIntBytes + kBBfBytes + 128;  // + TMEM address, 16 reduction words
constexpr uint32_t kBCols = 512;               // whole TMEM: 4 warps per lane quadrant x 128

// word of element u in the integer slice (a bijection on [0, 2^15))
__host__ __device__ constexpr int bf_swz(int u) { return u ^ (((u >> 4) & 3) << 3); }

// padded element index: non-decreasing pad (so the map is injective); the
// pass-2 accesses of a warp fall into 16 distinct banks
__host__ __device__ constexpr int bf_pad(int u) {
    return u + 2 * ((u >> 8) + 7 * (u >> 12));
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

template <bool F16>
__device__ __forceinline__ uint32_t pack16(float lo, float hi) {
    if constexpr (F16) {
        __half2 v = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&v);
    } else {
        __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&v);
    }
}

// one value rounded to the operand type, as its 16 bits
template <bool F16>
__device__ __forceinline__ uint16_t bits16(float x) {
    if constexpr (F16) {
        __half v = __float2half_rn(x);
        return *reinterpret_cast<uint16_t *>(&v);
    } else {
        __nv_bfloat16 v = __float2bfloat16_rn(x);
        return *reinterpret_cast<uint16_t *>(&v);
    }
}

__device__ __forceinline__ float hsign(int i, int j) {
    return (__popc(i & j) & 1) ? -1.f : 1.f;
}

// D (16x8, FP32) = A (16x16) . B (16x8), both operands BF16 or both FP16
template <bool F16>
__device__ __forceinline__ void mma16(float (&d)[4], const uint32_t (&a)[4],
                                      const uint32_t (&b)[2]) {
    if constexpr (F16)
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
            "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%10,%11,%12,%13};"
            : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "f"(0.f),
              "f"(0.f), "f"(0.f), "f"(0.f));
    else
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
            "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%10,%11,%12,%13};"
            : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "f"(0.f),
              "f"(0.f), "f"(0.f), "f"(0.f));
}

__device__ __forceinline__ void tmem_st8(uint32_t addr, const float (&x)[8]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n\t"
        "tcgen05.wait::st.sync.aligned;"
        :
        : "r"(addr), "r"(__float_as_uint(x[0])), "r"(__float_as_uint(x[1])),
          "r"(__float_as_uint(x[2])), "r"(__float_as_uint(x[3])), "r"(__float_as_uint(x[4])),
          "r"(__float_as_uint(x[5])), "r"(__float_as_uint(x[6])), "r"(__float_as_uint(x[7]))
        : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t addr, float (&x)[8]) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(addr)
        : "memory");
#pragma unroll
    for (int e = 0; e < 8; ++e) x[e] = __uint_as_float(r[e]);
}

// constant operand fragments of the Hadamard blocks for this lane
struct HFrags {
    uint32_t hA[4];      // H16 as the A operand (16x16)
    uint32_t hB[2][2];   // H16 as the B operand, columns 0-7 and 8-15
    uint32_t mB[2][2];   // H8 (x) I2 as the B operand: M[k][n] = H8[k>>1][n>>1] [k&1 == n&1]
};

__device__ __forceinline__ float m2(int k, int n) {
    return ((k & 1) == (n & 1)) ? hsign(k >> 1, n >> 1) : 0.f;
}

template <bool F16>
__device__ __forceinline__ void make_frags(HFrags &f, int g, int c) {
    // A fragment: (row g, k 2c..2c+1), (row g+8, k 2c..), (row g, k 2c+8..), (row g+8, k 2c+8..)
    f.hA[0] = pack16<F16>(hsign(g, 2 * c), hsign(g, 2 * c + 1));
    f.hA[1] = pack16<F16>(hsign(g + 8, 2 * c), hsign(g + 8, 2 * c + 1));
    f.hA[2] = pack16<F16>(hsign(g, 2 * c + 8), hsign(g, 2 * c + 9));
    f.hA[3] = pack16<F16>(hsign(g + 8, 2 * c + 8), hsign(g + 8, 2 * c + 9));
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int n = 8 * h + g;   // B fragment: (k 2c..2c+1, col n), (k 2c+8..2c+9, col n)
        f.hB[h][0] = pack16<F16>(hsign(2 * c, n), hsign(2 * c + 1, n));
        f.hB[h][1] = pack16<F16>(hsign(2 * c + 8, n), hsign(2 * c + 9, n));
        f.mB[h][0] = pack16<F16>(m2(2 * c, n), m2(2 * c + 1, n));
        f.mB[h][1] = pack16<F16>(m2(2 * c + 8, n), m2(2 * c + 9, n));
    }
}

// one tile: D2 = (H16 . X) . Bop for the two column halves.  xb[h] are the
// B-operand fragments of X (column half h); d2[h] the output fragments.
template <bool F16>
__device__ __forceinline__ void tile_pass(const HFrags &f, const uint32_t (&xb)[2][2],
                                          const uint32_t (&bop)[2][2], float (&d2)[2][4]) {
    float d1[2][4];
    mma16<F16>(d1[0], f.hA, xb[0]);
    mma16<F16>(d1[1], f.hA, xb[1]);
    // accumulator fragments of D1 = A-operand fragment of D1 (rows g / g+8, k = columns)
    const uint32_t a[4] = {pack16<F16>(d1[0][0], d1[0][1]), pack16<F16>(d1[0][2], d1[0][3]),
                           pack16<F16>(d1[1][0], d1[1][1]), pack16<F16>(d1[1][2], d1[1][3])};
    mma16<F16>(d2[0], a, bop[0]);
    mma16<F16>(d2[1], a, bop[1]);
}

// FP16 operands: the integer bucket sums enter as sum * 2^-27 (see the header)
constexpr float kF16In = 1.0f / 134217728.0f;    // 2^-27
constexpr float kF16Out = 134217728.0f;          // 2^27

// two integer bucket sums -> FP32 -> packed 16-bit pair: real values (sum *
// inv) for BF16, sum * 2^-27 for FP16
template <bool F16>
__device__ __forceinline__ uint32_t int2_to_16x2(int2 w, float inv) {
    const float sc = F16 ? kF16In : inv;
    return pack16<F16>(__int2float_rn(w.x) * sc, __int2float_rn(w.y) * sc);
}

// an FP32 transform output in real units (FP16: undo the 2^-27 and apply the
// column scale; two multiplies so that no factor overflows)
template <bool F16>
__device__ __forceinline__ float out_real(float v, float inv) {
    return F16 ? (v * kF16Out) * inv : v;
}

// the 2^15-point transform of the slice; `sink(i, vals)` receives, for the
// warp's i-th pass-2 tile, the 8 FP32 outputs of this thread.  Pass 1 reads
// (and clears) the integer slice Si, scaled by inv.
template <bool F16, typename Sink>
__device__ __forceinline__ void bf_fwht(int *Si, uint16_t *S16, const HFrags &f, int warp,
                                        int g, int c, float inv, Sink sink) {
    // pass 1: tiles tau = warp * 8 + i, u = a + 16 b + 256 tau
#pragma unroll 2
    for (int i = 0; i < kBTilesPerWarp; ++i) {
        const int tau = warp * kBTilesPerWarp + i;
        uint32_t xb[2][2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int b = 8 * h + g;
            const int u0 = 2 * c + 16 * b + 256 * tau;
            // elements (u0, u0 + 1) and (u0 + 8, u0 + 9), each pair read and
            // zeroed for the next scatter by one 64-bit exchange
            auto *p0 = reinterpret_cast<unsigned long long *>(Si + bf_swz(u0));
            auto *p1 = reinterpret_cast<unsigned long long *>(Si + bf_swz(u0 + 8));
            const unsigned long long r0 = atomicExch(p0, 0ull), r1 = atomicExch(p1, 0ull);
            const int2 w0 = make_int2((int)(uint32_t)r0, (int)(uint32_t)(r0 >> 32));
            const int2 w1 = make_int2((int)(uint32_t)r1, (int)(uint32_t)(r1 >> 32));
            xb[h][0] = int2_to_16x2<F16>(w0, inv);
            xb[h][1] = int2_to_16x2<F16>(w1, inv);
        }
        float d2[2][4];
        tile_pass<F16>(f, xb, f.hB, d2);
        // d2[h]: rows a' = g (regs 0,1) / g + 8 (regs 2,3), columns b' = 8h + 2c (+1)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
                const int ap = g + 8 * (rr >> 1);
                const int bp = 8 * h + 2 * c + (rr & 1);
                S16[bf_pad(ap + 16 * bp + 256 * tau)] = bits16<F16>(d2[h][rr]);
            }
        }
    }
    __syncthreads();
    // pass 2: tiles tau' = warp * 8 + i over bits 1-7, u = e + 2 tau' + 256 a2 + 4096 f
#pragma unroll 2
    for (int i = 0; i < kBTilesPerWarp; ++i) {
        const int taup = warp * kBTilesPerWarp + i;
        uint32_t xb[2][2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int n = 8 * h + g;
            const int e = n & 1, fq = n >> 1;
            const int base = e + 2 * taup + 4096 * fq;
            const int k0 = 2 * c;
            const int ua = base + 256 * k0, ub = base + 256 * (k0 + 1);
            const int uc = base + 256 * (k0 + 8), ud = base + 256 * (k0 + 9);
            const uint32_t va = S16[bf_pad(ua)], vb = S16[bf_pad(ub)];
            const uint32_t vc = S16[bf_pad(uc)], vd = S16[bf_pad(ud)];
            xb[h][0] = va | (vb << 16);
            xb[h][1] = vc | (vd << 16);
        }
        float d2[2][4];
        tile_pass<F16>(f, xb, f.mB, d2);
        float vals[8];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) vals[4 * h + rr] = out_real<F16>(d2[h][rr], inv);
        sink(i, vals);
    }
}

// index u (in the slice) of output value v (0..7) of pass-2 tile i for this thread
__device__ __forceinline__ int bf_out_index(int warp, int g, int c, int i, int v) {
    const int taup = warp * kBTilesPerWarp + i;
    const int h = v >> 2, rr = v & 3;
    const int a2 = g + 8 * (rr >> 1);
    const int n = 8 * h + 2 * c + (rr & 1);
    return (n & 1) + 2 * taup + 256 * a2 + 4096 * (n >> 1);
}

// one element of the fixed-point scatter: table word w (slice word in bits
// 0-14, sign in bit 15), sign applied by flipping the scale's sign bit
__device__ __forceinline__ void bf_scatter_one(int *Si, uint32_t w, float v, uint32_t sbits) {
    const float sc = __uint_as_float(sbits ^ ((w << 16) & 0x80000000u));
    atomicAdd(Si + (w & 0x7fffu), __float2int_rn(v * sc));
}

// scatter one column as integers round(v * s); all loads of a batch first
__device__ __forceinline__ void scatter_bf16(int *Si, const float *__restrict__ col,
                                             const tab_t *__restrict__ tab, int64_t n, int q,
                                             float s, int vec4) {
    const uint32_t sb = __float_as_uint(s);
    if (vec4) {   // n % 4 == 0, col 16-byte and tab 8-byte aligned
        constexpr int BV = 4;
        const float4 *c4 = reinterpret_cast<const float4 *>(col);
        const uint2 *t4 = reinterpret_cast<const uint2 *>(tab);
        const int64_t n4 = n >> 2;
        for (int64_t i = q; i < n4; i += BV * (int64_t)kBThreads) {
            float4 val[BV];
            uint2 w[BV];
#pragma unroll
            for (int e = 0; e < BV; ++e) {
                const bool ok = i + e * (int64_t)kBThreads < n4;
                val[e] = ok ? __ldcs(c4 + i + e * (int64_t)kBThreads) : make_float4(0.f, 0.f, 0.f, 0.f);
                w[e] = ok ? __ldg(t4 + i + e * (int64_t)kBThreads) : make_uint2(0u, 0u);
            }
#pragma unroll
            for (int e = 0; e < BV; ++e) {
                if (i + e * (int64_t)kBThreads < n4) {
                    bf_scatter_one(Si, w[e].x & 0xffffu, val[e].x, sb);
                    bf_scatter_one(Si, w[e].x >> 16, val[e].y, sb);
                    bf_scatter_one(Si, w[e].y & 0xffffu, val[e].z, sb);
                    bf_scatter_one(Si, w[e].y >> 16, val[e].w, sb);
                }
            }
        }
        return;
    }
    constexpr int B = 8;
    for (int64_t i = q; i < n; i += B * (int64_t)kBThreads) {
        float val[B];
        tab_t w[B];
#pragma unroll
        for (int e = 0; e < B; ++e) {
            const bool ok = i + e * (int64_t)kBThreads < n;
            val[e] = ok ? __ldcs(col + i + e * (int64_t)kBThreads) : 0.f;
            w[e] = ok ? __ldg(tab + i + e * (int64_t)kBThreads) : (tab_t)0;
        }
#pragma unroll
        for (int e = 0; e < B; ++e)
            if (i + e * (int64_t)kBThreads < n) bf_scatter_one(Si, w[e], val[e], sb);
    }
}

// largest number of table entries sharing a bucket (Si zero on entry and on
// return); all threads of the CTA
__device__ __forceinline__ int bf_cmax(int *Si, const tab_t *__restrict__ tab, int64_t n, int q,
                                       int *red) {
    for (int64_t i = q; i < n; i += kBThreads) atomicAdd(Si + (__ldg(tab + i) & 0x7fffu), 1);
    __syncthreads();
    int mx = 0;
    for (int i = q; i < kBN; i += kBThreads) {
        mx = max(mx, Si[i]);
        Si[i] = 0;
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((q & 31) == 0) red[q >> 5] = mx;
    __syncthreads();
    mx = 0;
#pragma unroll
    for (int w = 0; w < kBWarps; ++w) mx = max(mx, red[w]);
    __syncthreads();
    return mx;
}

// 2^e with cmax * colmax * 2^e < 2^30, e in [-126, 126]
__device__ __forceinline__ void bf_scale(float colmax, int cmax, float &s, float &inv) {
    const int Ec = ((__float_as_int(colmax) >> 23) & 0xff) - 126;
    const int Ek = 32 - __clz(cmax);
    const int e = min(max(30 - Ec - Ek, -126), 126);
    s = __int_as_float((127 + e) << 23);
    inv = __int_as_float((127 - e) << 23);
}

template <bool F16>
__global__ void __launch_bounds__(kBThreads, 1)
sketch_bf16_kernel(const float *__restrict__ At, int64_t ldat, const float *__restrict__ Bp,
                   int64_t ldbp, int64_t m, int64_t k, int64_t p, int Lfull, int C, int64_t chunk,
                   int d, const tab_t *__restrict__ tabA, const tab_t *__restrict__ tabB,
                   const float *__restrict__ colmax, double *__restrict__ partial, int vec4) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int *Si = reinterpret_cast<int *>(smem_raw);
    uint16_t *S = reinterpret_cast<uint16_t *>(smem_raw + kBIntBytes);
    uint32_t *s_taddr = reinterpret_cast<uint32_t *>(smem_raw + kBIntBytes + kBBfBytes);
    int *s_red = reinterpret_cast<int *>(smem_raw + kBIntBytes + kBBfBytes + 16);
    const int q = threadIdx.x, warp = q >> 5, lane = q & 31;
    const int g = lane >> 2, c = lane & 3;

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
    double *out = partial + (blk * d + r) * b + (int64_t)u_hi * kBN;

    if (warp == 0) {
        asm volatile(
            "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n\t"
            "tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;"
            :
            : "r"(smem_u32(s_taddr)), "r"(kBCols)
            : "memory");
    }
    for (int i = q; i < kBN; i += kBThreads) Si[i] = 0;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int cmaxA = bf_cmax(Si, tA, m, q, s_red);
    const int cmaxB = bf_cmax(Si, tB, p, q, s_red);
    // lanes of quadrant warp % 4; four warps share a quadrant: columns 128 * (warp / 4) ...
    const uint32_t tx = *s_taddr + ((uint32_t)(32 * (warp & 3)) << 16) + 128u * (uint32_t)(warp >> 2);
    const uint32_t tz = tx + 64;
    HFrags f;
    make_frags<F16>(f, g, c);
    {
        float zero[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) zero[e] = 0.f;
#pragma unroll
        for (int i = 0; i < kBTilesPerWarp; ++i) tmem_st8(tz + 8 * i, zero);
    }

    for (int64_t t = t0; t < t1; ++t) {
        float sA, invA, sB, invB;
        bf_scale(__ldg(colmax + t), cmaxA, sA, invA);
        bf_scale(__ldg(colmax + k + t), cmaxB, sB, invB);
        scatter_bf16(Si, At + t * ldat, tA, m, q, sA, vec4);
        __syncthreads();
        bf_fwht<F16>(Si, S, f, warp, g, c, invA,
                [&](int i, const float(&vals)[8]) { tmem_st8(tx + 8 * i, vals); });
        __syncthreads();
        scatter_bf16(Si, Bp + t * ldbp, tB, p, q, sB, vec4);
        __syncthreads();
        bf_fwht<F16>(Si, S, f, warp, g, c, invB, [&](int i, const float(&vals)[8]) {
            float xs[8], zs[8];
            tmem_ld8(tx + 8 * i, xs);
            tmem_ld8(tz + 8 * i, zs);
#pragma unroll
            for (int e = 0; e < 8; ++e) zs[e] = fmaf(xs[e], vals[e], zs[e]);
            tmem_st8(tz + 8 * i, zs);
        });
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < kBTilesPerWarp; ++i) {
        float zs[8];
        tmem_ld8(tz + 8 * i, zs);
#pragma unroll
        for (int v = 0; v < 8; ++v) out[bf_out_index(warp, g, c, i, v)] = (double)zs[v];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :
                     : "r"(*s_taddr), "r"(kBCols)
                     : "memory");
    }
}

// scatter words for the integer slice: word of the bucket | sign << 15
__global__ void bf16_table_kernel(const __grid_constant__ HashParams hp, int d, int Lfull, int C,
                                  int64_t m, int64_t p, tab_t *__restrict__ tabA,
                                  tab_t *__restrict__ tabB) {
    const int shift = 64 - Lfull;
    const int64_t nA = (int64_t)d * C * m, n = nA + (int64_t)d * C * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const bool isA = e < nA;
        const int64_t fidx = isA ? e : e - nA;
        const int64_t len = isA ? m : p;
        const int64_t slot = fidx / len;
        const uint64_t x = (uint64_t)(fidx % len);
        const int r = (int)(slot / C);
        const uint32_t u_hi = (uint32_t)(slot % C);
        const HashRep &H = hp.rep[r];
        const uint32_t h = isA ? mas_hash(H.a1, H.c1, x, shift) : mas_hash(H.a2, H.c2, x, shift);
        const uint32_t sb = isA ? mas_sign_bit(H.as1, H.cs1, x) : mas_sign_bit(H.as2, H.cs2, x);
        const uint32_t neg = sb ^ (__popc((h >> kBL) & u_hi) & 1u);
        const tab_t w = (tab_t)((uint32_t)bf_swz((int)(h & (kBN - 1))) | (neg << 15));
        if (isA)
            tabA[fidx] = w;
        else
            tabB[fidx] = w;
    }
}

}  // namespace

int sketch_bf16_llo() { return kBL; }
int sketch_bf16_threads() { return kBThreads; }
size_t sketch_bf16_smem() { return kBSmem; }

cudaError_t launch_sketch_bf16(const SketchPlan &pl, const float *At, const float *Bp, int64_t m,
                               int64_t k, int64_t p, int d, const HashParams &hp, tab_t *tabA,
                               tab_t *tabB, const float *colmax, double *partial, bool f16,
                               cudaStream_t s) {
    const int64_t n = (int64_t)d * pl.C * (m + p);
    int64_t gsz = (n + 255) / 256;
    if (gsz > 152 * 32) gsz = 152 * 32;
    if (gsz < 1) gsz = 1;
    bf16_table_kernel<<<(unsigned)gsz, 256, 0, s>>>(hp, d, pl.L, pl.C, m, p, tabA, tabB);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto kern = f16 ? sketch_bf16_kernel<true> : sketch_bf16_kernel<false>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBSmem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (int64_t)pl.nchunks * d * pl.C;
    const bool vec4 = m % 4 == 0 && p % 4 == 0 && pl.ldat % 4 == 0 && pl.ldbp % 4 == 0 &&
                      reinterpret_cast<uintptr_t>(At) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(Bp) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(tabA) % 8 == 0 &&
                      reinterpret_cast<uintptr_t>(tabB) % 8 == 0;
    kern<<<(unsigned)blocks, kBThreads, kBSmem, s>>>(
        At, pl.ldat, Bp, pl.ldbp, m, k, p, pl.L, pl.C, pl.chunk, d, tabA, tabB, colmax, partial,
        vec4 ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace cmm
