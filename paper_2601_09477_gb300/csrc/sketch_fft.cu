// sketch_fft.cu -- the sketch of Pagh's original form (Sec. 3.1): the same
// sketches x_t, y_t as Algorithm 1, but the product polynomial is the cyclic
// convolution of Sec. 2, R_r = sum_t x_t * y_t, computed through the FFT:
// R_r = (1/b) IDFT( sum_t DFT(x_t) o DFT(y_t) ), DFT[k] = sum_n x[n] w_b^{nk},
// w_b = exp(-2 pi i / b).  Estimates then read bucket h1(i) + h2(j) mod b.
//
// Work decomposition (FP32 butterflies, slices of N = 2^13 frequencies):
// b = C N and the CTA for class c in [0, C) owns the frequencies k = c + C k'
// (k' < N):
//     X[c + C k'] = DFT_N(f_c)[k'],
//     f_c[n] = w_b^{c n} sum_{h_hi} w_C^{c h_hi} x[n + N h_hi],
// so the scatter adds each value, times the C-th root of unity w_C^{c h_hi(i)},
// into the complex slot h_lo(i) -- no exchange between CTAs (the analogue of
// the frequency split of the FWHT kernels).  x is real, so class C - c holds
// the conjugates of class c (X[b - k] = conj X[k]); only classes 0 .. C/2 run.
//
// The N-point transform is a four-step FFT, 8192 = 32 x 32 x 8, with 256
// threads of 32 complex values each:
//   round 0: thread q holds f[q + 256 j], j < 32 (times the class factor
//            w_b^{c (q + 256 j)}); a 32-point DFT over j, then the twiddle
//            w_N^{q k1};
//   round 1: thread (q_lo, r0) holds the values of q = q_lo + 8 q_hi; a 32-point
//            DFT over q_hi, then the twiddle w_256^{q_lo k1'};
//   round 2: four 8-point DFTs over q_lo.
// The register DFTs are radix-2 decimation-in-frequency (bit-reversed output)
// with exact constant twiddles; frequency k' = k1 + 32 (k1' + 32 k2) of every
// (thread, register) is tracked and used when the CTA writes its partial.
// Slot u lives at complex word u + (u >> 4) + 8 (u >> 8): the 64-bit accesses
// of all three rounds are bank-conflict free.
//
// The scatter is the fixed-point integer scatter of the FWHT kernels (both
// components of the weighted value as integers at the column's power-of-two
// scale), X is kept in TMEM and Z = sum_t X o Y accumulates there in FP32; each
// CTA writes its FP64 partial (complex, natural frequency order).  The finish
// (FP64): per class an inverse N-point DFT g_c, then
//     R[w] = (1/b) Re sum_c w_b^{-w c} g_c[w mod N].
#include "cmm_internal.h"
#include "fwht_device.cuh"
#include "sketch_impl.cuh"

namespace cmm {

namespace {

constexpr int kFL = 13;
constexpr int kFN = 1 << kFL;
constexpr int kFT = 256;                 // threads per CTA
constexpr int kFE = 32;                  // complex values per thread
constexpr int kFStride = 8960;           // padded slice in complex words
constexpr int kFMaxC = 1 << (CMM_MAX_LOG2B - kFL);
constexpr uint32_t kFCols = 256;         // TMEM: 64 columns X + 64 columns Z, two warps per lane quadrant

__host__ __device__ constexpr int fpad(int u) { return u + (u >> 4) + 8 * (u >> 8); }
static_assert(fpad(kFN - 1) < kFStride, "padded slice");

// shared memory: slice | w_N^e (e < 128) | w_N^{128 e} (e < 64) | w_256^e |
// class factors | scatter weights w_C^e | TMEM address and reduction words
constexpr size_t kFOffLo = (size_t)kFStride * 8;
constexpr size_t kFOffHi = kFOffLo + 128 * 8;
constexpr size_t kFOff256 = kFOffHi + 64 * 8;
constexpr size_t kFOffSig = kFOff256 + 256 * 8;
constexpr size_t kFOffW = kFOffSig + 32 * 8;
constexpr size_t kFOffCtl = kFOffW + (size_t)kFMaxC * 8;
constexpr size_t kFSmem = kFOffCtl + 64;

// cos(pi e / 16), e = 0 .. 8
__device__ constexpr float kCos16[9] = {1.0f,
                                        0.98078528040323043f,
                                        0.92387953251128674f,
                                        0.83146961230254524f,
                                        0.70710678118654752f,
                                        0.55557023301960218f,
                                        0.38268343236508977f,
                                        0.19509032201612826f,
                                        0.0f};

// (re, im) *= w_32^e = exp(-2 pi i e / 32), 0 <= e < 16 (e is a compile-time
// constant after unrolling, so only one branch survives)
__device__ __forceinline__ void mul_w32(int e, float &re, float &im) {
    if (e == 0) return;
    if (e == 8) {   // -i
        const float t = re;
        re = im;
        im = -t;
        return;
    }
    if (e == 4) {   // (1 - i) / sqrt 2
        const float c = kCos16[4];
        const float t = (re + im) * c;
        im = (im - re) * c;
        re = t;
        return;
    }
    if (e == 12) {   // (-1 - i) / sqrt 2
        const float c = kCos16[4];
        const float t = (im - re) * c;
        im = -(re + im) * c;
        re = t;
        return;
    }
    const float wr = e < 8 ? kCos16[e] : -kCos16[16 - e];
    const float wi = -(e < 8 ? kCos16[8 - e] : kCos16[e - 8]);
    const float t = fmaf(re, wr, -im * wi);
    im = fmaf(re, wi, im * wr);
    re = t;
}

// in-place DFT of length LEN (32 or 8) on re/im[OFF .. OFF+LEN): radix-2
// decimation in frequency, natural order in, bit-reversed order out
template <int LEN, int OFF, int NV>
__device__ __forceinline__ void dft_dif(float (&re)[NV], float (&im)[NV]) {
#pragma unroll
    for (int h = LEN / 2; h >= 1; h >>= 1) {
#pragma unroll
        for (int j = 0; j < LEN; ++j) {
            if (j & h) continue;
            const float ar = re[OFF + j], ai = im[OFF + j];
            const float br = re[OFF + j + h], bi = im[OFF + j + h];
            re[OFF + j] = ar + br;
            im[OFF + j] = ai + bi;
            float dr = ar - br, di = ai - bi;
            mul_w32((j % h) * (16 / h), dr, di);   // w_{2h}^{j mod h}
            re[OFF + j + h] = dr;
            im[OFF + j + h] = di;
        }
    }
}

__device__ __forceinline__ int brev5(int x) { return (int)(__brev((unsigned)x) >> 27); }
__device__ __forceinline__ int brev3(int x) { return (int)(__brev((unsigned)x) >> 29); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ uint32_t f_smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void f_tmem_st16(uint32_t addr, const float *x) {
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

__device__ __forceinline__ void f_tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void f_tmem_ld16(uint32_t addr, float (&x)[16]) {
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

// one element of the complex fixed-point scatter: table word w = padded slot
// (bits 0-13) | sign (bit 14) | exponent of the weight w_C^e (bits 15-25)
__device__ __forceinline__ void fscatter_one(int *Si, const float2 *Wc, uint32_t w, float v,
                                             float s) {
    const float2 wt = Wc[w >> 15];
    const float val = ((w >> 14) & 1u) ? -v * s : v * s;
    int *slot = Si + 2 * (w & 0x3fffu);
    if (wt.x != 0.f) atomicAdd(slot, __float2int_rn(val * wt.x));
    if (wt.y != 0.f) atomicAdd(slot + 1, __float2int_rn(val * wt.y));
}

// scatter one column; all loads of a batch issued before its atomics
__device__ __forceinline__ void fscatter(int *Si, const float2 *Wc, const float *__restrict__ col,
                                         const uint32_t *__restrict__ tab, int64_t n, int q,
                                         float s) {
    constexpr int B = 16;
    for (int64_t i = q; i < n; i += B * (int64_t)kFT) {
        float val[B];
        uint32_t w[B];
#pragma unroll
        for (int e = 0; e < B; ++e) {
            const bool ok = i + e * (int64_t)kFT < n;
            val[e] = ok ? __ldcs(col + i + e * (int64_t)kFT) : 0.f;
            w[e] = ok ? __ldg(tab + i + e * (int64_t)kFT) : 0u;
        }
#pragma unroll
        for (int e = 0; e < B; ++e)
            if (i + e * (int64_t)kFT < n) fscatter_one(Si, Wc, w[e], val[e], s);
    }
}

// the N-point transform of the slice (complex integer sums scaled by inv) for
// class c; result: re/im[8 jg + r2] = frequency fk(q, jg, r2).  The slice is
// left zeroed.
__device__ __forceinline__ void fft_slice(float2 *S, const float2 *tlo, const float2 *thi,
                                          const float2 *t256, const float2 *sig, float2 rho,
                                          bool shifted, int q, float inv, float (&re)[kFE],
                                          float (&im)[kFE]) {
    const int2 *Si2 = reinterpret_cast<const int2 *>(S);
    // round 0
#pragma unroll
    for (int j = 0; j < kFE; ++j) {
        const int2 w = Si2[fpad(q + 256 * j)];
        re[j] = __int2float_rn(w.x) * inv;
        im[j] = __int2float_rn(w.y) * inv;
    }
    if (shifted) {
#pragma unroll
        for (int j = 0; j < kFE; ++j) {
            const float2 v = cmul(make_float2(re[j], im[j]), sig[j]);
            re[j] = v.x;
            im[j] = v.y;
        }
    }
    dft_dif<32, 0, kFE>(re, im);
#pragma unroll
    for (int r = 0; r < kFE; ++r) {
        const int e = q * brev5(r);   // < 8192
        float2 tw = cmul(tlo[e & 127], thi[e >> 7]);
        if (shifted) tw = cmul(tw, rho);
        const float2 v = cmul(make_float2(re[r], im[r]), tw);
        S[fpad(q + 256 * r)] = v;
    }
    __syncthreads();
    // round 1
    {
        const int ql = q & 7, r0 = q >> 3;
#pragma unroll
        for (int j = 0; j < kFE; ++j) {
            const float2 v = S[fpad(ql + 8 * j + 256 * r0)];
            re[j] = v.x;
            im[j] = v.y;
        }
        dft_dif<32, 0, kFE>(re, im);
#pragma unroll
        for (int r = 0; r < kFE; ++r)
            S[fpad(ql + 8 * r + 256 * r0)] = cmul(make_float2(re[r], im[r]), t256[ql * brev5(r)]);
    }
    __syncthreads();
    // round 2
#pragma unroll
    for (int jg = 0; jg < 4; ++jg) {
        const int g = q + 256 * jg;
#pragma unroll
        for (int l = 0; l < 8; ++l) {
            // read and zeroed for the next scatter by one 64-bit exchange
            auto *p = reinterpret_cast<unsigned long long *>(S + fpad(8 * g + l));
            const unsigned long long v = atomicExch(p, 0ull);
            re[8 * jg + l] = __uint_as_float((uint32_t)v);
            im[8 * jg + l] = __uint_as_float((uint32_t)(v >> 32));
        }
    }
    dft_dif<8, 0, kFE>(re, im);
    dft_dif<8, 8, kFE>(re, im);
    dft_dif<8, 16, kFE>(re, im);
    dft_dif<8, 24, kFE>(re, im);
}

// frequency (within the class) of register 8 jg + r2 of thread q after fft_slice
__device__ __forceinline__ int fk(int q, int jg, int r2) {
    const int g = q + 256 * jg;
    return brev5(g >> 5) + 32 * brev5(g & 31) + 1024 * brev3(r2);
}

__global__ void __launch_bounds__(kFT, 2)
sketch_fft_kernel(const float *__restrict__ At, int64_t ldat, const float *__restrict__ Bp,
                  int64_t ldbp, int64_t m, int64_t k, int64_t p, int Lfull, int C, int NC,
                  int64_t chunk, int d, const uint32_t *__restrict__ tabA,
                  const uint32_t *__restrict__ tabB, const float *__restrict__ colmax,
                  double *__restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *S = reinterpret_cast<float2 *>(smem_raw);
    int *Si = reinterpret_cast<int *>(smem_raw);
    float2 *tlo = reinterpret_cast<float2 *>(smem_raw + kFOffLo);
    float2 *thi = reinterpret_cast<float2 *>(smem_raw + kFOffHi);
    float2 *t256 = reinterpret_cast<float2 *>(smem_raw + kFOff256);
    float2 *sig = reinterpret_cast<float2 *>(smem_raw + kFOffSig);
    float2 *Wc = reinterpret_cast<float2 *>(smem_raw + kFOffW);
    uint32_t *s_taddr = reinterpret_cast<uint32_t *>(smem_raw + kFOffCtl);
    int *s_red = reinterpret_cast<int *>(smem_raw + kFOffCtl + 16);
    const int q = threadIdx.x, warp = q >> 5;

    int item = blockIdx.x;
    const int ci = item % NC;        // class c = ci (0 .. C/2)
    item /= NC;
    const int r = item % d;
    const int64_t blk = item / d;
    const int64_t t0 = blk * chunk;
    const int64_t t1 = (t0 + chunk < k) ? t0 + chunk : k;
    const int64_t slot = (int64_t)r * NC + ci;
    const uint32_t *tA = tabA + slot * m;
    const uint32_t *tB = tabB + slot * p;
    double *out = partial + (((int64_t)blk * d + r) * NC + ci) * (2 * (int64_t)kFN);
    const double b = (double)((int64_t)1 << Lfull);

    if (warp == 0) {
        asm volatile(
            "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n\t"
            "tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;"
            :
            : "r"(f_smem_addr(s_taddr)), "r"(kFCols)
            : "memory");
    }
    // tables: w_N^e, w_N^{128 e}, w_256^e, class factors w_b^{256 c j}, w_C^e
    for (int e = q; e < 128; e += kFT) {
        float sn, cs;
        sincospif(-2.0f * (float)e / (float)kFN, &sn, &cs);
        tlo[e] = make_float2(cs, sn);
    }
    for (int e = q; e < 64; e += kFT) {
        float sn, cs;
        sincospif(-2.0f * (float)(128 * e) / (float)kFN, &sn, &cs);
        thi[e] = make_float2(cs, sn);
    }
    for (int e = q; e < 256; e += kFT) {
        float sn, cs;
        sincospif(-2.0f * (float)e / 256.0f, &sn, &cs);
        t256[e] = make_float2(cs, sn);
    }
    for (int j = q; j < 32; j += kFT) {
        // w_b^{256 c j}: exponent 2 (256 c j mod b) / b, exact in FP64
        const double ex = (double)(((int64_t)256 * ci * j) & ((int64_t)b - 1)) / b;
        double sn, cs;
        sincospi(-2.0 * ex, &sn, &cs);
        sig[j] = make_float2((float)cs, (float)sn);
    }
    for (int e = q; e < C; e += kFT) {
        const double ex = (double)e / (double)C;
        double sn, cs;
        sincospi(-2.0 * ex, &sn, &cs);
        // exact zeros keep the scatter of real (or imaginary) weights to one atomic
        Wc[e] = make_float2((float)cs, (float)sn);
    }
    for (int i = q; i < 2 * kFStride; i += kFT) Si[i] = 0;
    float2 rho;
    {
        // w_b^{c q}
        const double ex = (double)(((int64_t)ci * q) & ((int64_t)b - 1)) / b;
        double sn, cs;
        sincospi(-2.0 * ex, &sn, &cs);
        rho = make_float2((float)cs, (float)sn);
    }
    const bool shifted = ci != 0;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // bucket occupancy of this repetition (slot field of the tables)
    int cmaxA, cmaxB;
    {
        int mx[2];
        for (int h = 0; h < 2; ++h) {
            const uint32_t *tab = h ? tB : tA;
            const int64_t n = h ? p : m;
            for (int64_t i = q; i < n; i += kFT) atomicAdd(Si + 2 * (__ldg(tab + i) & 0x3fffu), 1);
            __syncthreads();
            int v = 0;
            for (int i = q; i < kFStride; i += kFT) {
                v = max(v, Si[2 * i]);
                Si[2 * i] = 0;
            }
            v = __reduce_max_sync(0xffffffffu, v);
            if ((q & 31) == 0) s_red[q >> 5] = v;
            __syncthreads();
            v = 0;
#pragma unroll
            for (int w = 0; w < kFT / 32; ++w) v = max(v, s_red[w]);
            mx[h] = v;
            __syncthreads();
        }
        cmaxA = mx[0];
        cmaxB = mx[1];
    }
    const uint32_t tx = *s_taddr + ((uint32_t)(32 * (warp & 3)) << 16) + 128u * (uint32_t)(warp >> 2);
    const uint32_t tz = tx + 64;
    {
        float zero[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) zero[e] = 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) f_tmem_st16(tz + 16 * c, zero);
        f_tmem_wait_st();
    }

    float re[kFE], im[kFE];
    for (int64_t t = t0; t < t1; ++t) {
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            float sc, inv;
            fixed_scale(__ldg(colmax + (half ? k : 0) + t), half ? cmaxB : cmaxA, sc, inv);
            if (half == 0)
                fscatter(Si, Wc, At + t * ldat, tA, m, q, sc);
            else
                fscatter(Si, Wc, Bp + t * ldbp, tB, p, q, sc);
            __syncthreads();
            fft_slice(S, tlo, thi, t256, sig, rho, shifted, q, inv, re, im);
            if (half == 0) {
                f_tmem_st16(tx, re);
                f_tmem_st16(tx + 16, re + 16);
                f_tmem_st16(tx + 32, im);
                f_tmem_st16(tx + 48, im + 16);
            } else {
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    float xr[16], xi[16], zr[16], zi[16];
                    f_tmem_ld16(tx + 16 * c, xr);
                    f_tmem_ld16(tx + 32 + 16 * c, xi);
                    f_tmem_ld16(tz + 16 * c, zr);
                    f_tmem_ld16(tz + 32 + 16 * c, zi);
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const float yr = re[16 * c + e], yi = im[16 * c + e];
                        zr[e] = fmaf(xr[e], yr, fmaf(-xi[e], yi, zr[e]));
                        zi[e] = fmaf(xr[e], yi, fmaf(xi[e], yr, zi[e]));
                    }
                    f_tmem_st16(tz + 16 * c, zr);
                    f_tmem_st16(tz + 32 + 16 * c, zi);
                }
            }
            f_tmem_wait_st();
            __syncthreads();
        }
    }

    // partial: Z of this class, complex FP64, natural frequency order
    {
        float zr[16], zi[16];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            f_tmem_ld16(tz + 16 * c, zr);
            f_tmem_ld16(tz + 32 + 16 * c, zi);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int v = 16 * c + e;
                const int kk = fk(q, v >> 3, v & 7);
                out[2 * kk] = (double)zr[e];
                out[2 * kk + 1] = (double)zi[e];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :
                     : "r"(*s_taddr), "r"(kFCols)
                     : "memory");
    }
}

// table word per (r, class, element): padded slot | sign << 14 | (c h_hi mod C) << 15
__global__ void fft_table_kernel(const __grid_constant__ HashParams hp, int d, int Lfull, int C,
                                 int NC, int64_t m, int64_t p, uint32_t *__restrict__ tabA,
                                 uint32_t *__restrict__ tabB) {
    const int shift = 64 - Lfull;
    const int64_t nA = (int64_t)d * NC * m, n = nA + (int64_t)d * NC * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const bool isA = e < nA;
        const int64_t f = isA ? e : e - nA;
        const int64_t len = isA ? m : p;
        const int64_t slot = f / len;
        const uint64_t x = (uint64_t)(f % len);
        const int r = (int)(slot / NC);
        const uint32_t c = (uint32_t)(slot % NC);
        const HashRep &H = hp.rep[r];
        const uint32_t h = isA ? mas_hash(H.a1, H.c1, x, shift) : mas_hash(H.a2, H.c2, x, shift);
        const uint32_t sb = isA ? mas_sign_bit(H.as1, H.cs1, x) : mas_sign_bit(H.as2, H.cs2, x);
        const uint32_t wexp = (c * (h >> kFL)) & (uint32_t)(C - 1);
        const uint32_t w = (uint32_t)fpad((int)(h & (kFN - 1))) | (sb << 14) | (wexp << 15);
        if (isA)
            tabA[f] = w;
        else
            tabB[f] = w;
    }
}

// ---- FP64 finish ----------------------------------------------------------
constexpr int kFFinThreads = 512;
constexpr size_t kFFinSmem = (size_t)kFN * 16 + (size_t)(kFN / 2) * 16;

// per (r, class c in [0, C)): Z_c = sum over blocks (classes above C/2 from
// the conjugates of class C - c), then g_c = the unnormalised inverse DFT of
// length N, written to G[r][c][n] (complex FP64)
__global__ void __launch_bounds__(kFFinThreads, 1)
fft_finish_class_kernel(const double *__restrict__ partial, int nchunks, int d, int C, int NC,
                        double *__restrict__ G) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *Z = reinterpret_cast<double2 *>(smem_raw);
    double2 *tw = reinterpret_cast<double2 *>(smem_raw + (size_t)kFN * 16);
    const int r = blockIdx.x / C, c = blockIdx.x % C;
    const bool conj = 2 * c > C;
    const int cs = conj ? C - c : c;
    for (int e = threadIdx.x; e < kFN / 2; e += kFFinThreads) {
        double sn, csn;
        sincospi(2.0 * (double)e / (double)kFN, &sn, &csn);   // inverse: exp(+2 pi i e / N)
        tw[e] = make_double2(csn, sn);
    }
    const int64_t stride = (int64_t)d * NC * 2 * kFN;
    const double *src = partial + ((int64_t)r * NC + cs) * 2 * kFN;
    for (int kk = threadIdx.x; kk < kFN; kk += kFFinThreads) {
        const int ks = conj ? kFN - 1 - kk : kk;
        double zr = 0.0, zi = 0.0;
        for (int blk = 0; blk < nchunks; ++blk) {
            zr += src[blk * stride + 2 * ks];
            zi += src[blk * stride + 2 * ks + 1];
        }
        Z[kk] = make_double2(zr, conj ? -zi : zi);
    }
    __syncthreads();
    // radix-2 decimation in frequency: natural order in, bit-reversed out
    for (int h = kFN / 2; h >= 1; h >>= 1) {
        for (int i = threadIdx.x; i < kFN / 2; i += kFFinThreads) {
            const int jlo = i % h;
            const int j = (i / h) * 2 * h + jlo;
            const double2 a = Z[j], bb = Z[j + h];
            const double2 w = tw[jlo * (kFN / (2 * h))];
            const double dr = a.x - bb.x, di = a.y - bb.y;
            Z[j] = make_double2(a.x + bb.x, a.y + bb.y);
            Z[j + h] = make_double2(dr * w.x - di * w.y, dr * w.y + di * w.x);
        }
        __syncthreads();
    }
    double2 *g = reinterpret_cast<double2 *>(G) + ((int64_t)r * C + c) * kFN;
    for (int pos = threadIdx.x; pos < kFN; pos += kFFinThreads)
        g[(int)(__brev((unsigned)pos) >> (32 - kFL))] = Z[pos];
}

// R[r][w] = (1/b) Re sum_c w_b^{-w c} g_c[w mod N]
__global__ void fft_finish_combine_kernel(const double *__restrict__ G, int d, int L, int C,
                                          double *__restrict__ R) {
    const int64_t b = (int64_t)1 << L;
    const double inv_b = ldexp(1.0, -L);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)d * b;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e >> L);
        const int64_t w = e & (b - 1);
        const double2 *g = reinterpret_cast<const double2 *>(G) + (int64_t)r * C * kFN + (w & (kFN - 1));
        double sn, cs;
        sincospi(2.0 * (double)w / (double)b, &sn, &cs);
        double pr = 1.0, pi = 0.0, acc = 0.0;
        for (int c = 0; c < C; ++c) {
            const double2 v = g[(int64_t)c * kFN];
            acc += pr * v.x - pi * v.y;
            const double t = pr * cs - pi * sn;
            pi = pr * sn + pi * cs;
            pr = t;
            if ((c & 63) == 63) {   // re-anchor the power every 64 steps
                double s2, c2;
                sincospi(2.0 * (double)(((int64_t)(c + 1) * w) & (b - 1)) / (double)b, &s2, &c2);
                pr = c2;
                pi = s2;
            }
        }
        R[e] = acc * inv_b;
    }
}

}  // namespace

int sketch_fft_llo() { return kFL; }
int sketch_fft_threads() { return kFT; }
size_t sketch_fft_smem() { return kFSmem; }

cudaError_t launch_sketch_fft(const SketchPlan &pl, const float *At, const float *Bp, int64_t m,
                              int64_t k, int64_t p, int d, const HashParams &hp, uint32_t *tabA,
                              uint32_t *tabB, const float *colmax, double *partial,
                              cudaStream_t s) {
    const int C = pl.C, NC = pl.nclass;
    {
        const int64_t n = (int64_t)d * NC * (m + p);
        int64_t g = (n + 255) / 256;
        if (g > 152 * 32) g = 152 * 32;
        if (g < 1) g = 1;
        fft_table_kernel<<<(unsigned)g, 256, 0, s>>>(hp, d, pl.L, C, NC, m, p, tabA, tabB);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaFuncSetAttribute(sketch_fft_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFSmem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (int64_t)pl.nchunks * d * NC;
    sketch_fft_kernel<<<(unsigned)blocks, kFT, kFSmem, s>>>(At, pl.ldat, Bp, pl.ldbp, m, k, p,
                                                            pl.L, C, NC, pl.chunk, d, tabA, tabB,
                                                            colmax, partial);
    return cudaGetLastError();
}

cudaError_t launch_finish_fft(const double *partial, int nchunks, int d, int L, int C, int NC,
                              double *G, double *R, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(fft_finish_class_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFFinSmem);
    if (e != cudaSuccess) return e;
    fft_finish_class_kernel<<<(unsigned)(d * C), kFFinThreads, kFFinSmem, s>>>(partial, nchunks, d,
                                                                              C, NC, G);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t n = (int64_t)d << L;
    int64_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    fft_finish_combine_kernel<<<(unsigned)g, 256, 0, s>>>(G, d, L, C, R);
    return cudaGetLastError();
}

}  // namespace cmm
