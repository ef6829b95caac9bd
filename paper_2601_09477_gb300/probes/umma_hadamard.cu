// umma_hadamard.cu -- cost of the 2^14-point Walsh-Hadamard transform of one
// slice done on the fifth-generation tensor cores, on the device it runs on:
// the slice as a 128 x 128 matrix X (x[128 k + n] = X[k][n]) transforms as
// Y = H128 X H128, two M = N = K = 128 products with BF16 operands and FP32
// accumulation (tcgen05.mma, kind::f16): D1 = H X with H in tensor memory
// (TMEM) as the A operand and X in shared memory as the B operand, D1
// rounded to BF16 into TMEM by the threads, then Y = D1 H with D1 from TMEM
// and H from shared memory.  Y[i][j] is the transform at index 128 i + j.
//
// Modes (one CTA of 512 threads per SM, each looping over `iters` slices):
//   0  the two products only (the intermediate is not rewritten)
//   1  the products and the TMEM -> register -> TMEM rounding of D1
//   2  as 1, plus the shared-memory pass the sketch would add per slice: the
//      integer bucket sums (2^14 words) read, cleared and written as the BF16
//      B operand (32 KiB) before the first product
// Per slice it reports SM clocks, and the tensor rate as FP32 FLOP/s of the
// products (2 x 2 x 128^3 per slice).  With iters = 1, CTA 0's Y is written
// out and checked by the host against the exact transform of a {-1, 0, 1}
// slice (every value stays an integer below 2^8 before the BF16 rounding, so
// Y is exact).
//
// Bounds: shared memory holds the integer slice (64 KiB), X (32 KiB), H
// (32 KiB) and one mbarrier; every descriptor addresses only the X or H
// region (K-major, core matrix (r, c) of 128 bytes at ((c * 16 + r) * 128),
// leading-dimension offset 2048, stride-dimension offset 128; k-block kb
// starts at kb * 4096); TMEM columns [0, 256) are allocated and used as H
// [0, 64), D1 and Y [64, 192), the BF16 D1 [192, 256).  All waits are bounded
// and report through `status`.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include <cuda_runtime.h>

#include "../csrc/tmem_device.cuh"
#include "../csrc/umma_device.cuh"

#define CHECK(x)                                                                     \
    do {                                                                             \
        cudaError_t e_ = (x);                                                        \
        if (e_ != cudaSuccess) {                                                     \
            std::fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));            \
            return 1;                                                                \
        }                                                                            \
    } while (0)

namespace {

constexpr int kThreads = 512;
constexpr int kSliceBytes = 1 << 16;           // 2^14 int32 bucket sums
constexpr int kOpBytes = 128 * 128 * 2;        // one BF16 operand
constexpr int kSmem = kSliceBytes + 2 * kOpBytes + 16;
constexpr uint32_t kCols = 256;
constexpr uint32_t kWaitPolls = 1u << 22;

// byte offset of element (row r, k) of a 128 x 128 K-major BF16 operand
__host__ __device__ constexpr uint32_t op_off(int r, int k) {
    return (uint32_t)(((k >> 3) * 16 + (r >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// word of slice point u = 128 k + n in the integer slice: the 8 values of one
// 16-byte operand chunk (same n, k = 8 kc .. 8 kc + 7) are contiguous
__host__ __device__ constexpr int slice_word(int u) {
    return ((((u >> 7) >> 3) * 128 + (u & 127)) << 3) | ((u >> 7) & 7);
}

__device__ __forceinline__ int hsign(int i, int k) { return (__popc(i & k) & 1) ? -1 : 1; }

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// integer bucket sum (|x| < 2^22) to FP32 without a conversion instruction
__device__ __forceinline__ float int22_to_f(int x) {
    return __int_as_float(0x4B400000 + x) - 12582912.f;
}

__device__ unsigned long long g_clk;

__global__ void __launch_bounds__(kThreads, 1)
umma_hadamard(int mode, int iters, const int8_t *__restrict__ x0, float *__restrict__ yout,
              int *__restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t s_taddr;
    int *slice = reinterpret_cast<int *>(smem);
    unsigned char *xop = smem + kSliceBytes;
    unsigned char *hop = xop + kOpBytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(hop + kOpBytes);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) cmm::tm::alloc(&s_taddr, kCols);
    // the slice (CTA 0: the host's values; others: a pattern), H in shared memory
    for (int u = tid; u < 128 * 128; u += kThreads) {
        const int v = blockIdx.x == 0 ? (int)x0[u] : ((u * 7 + blockIdx.x) % 3) - 1;
        slice[slice_word(u)] = v;
        const int r = u & 127, k = u >> 7;
        *reinterpret_cast<uint16_t *>(hop + op_off(r, k)) = hsign(r, k) > 0 ? 0x3F80 : 0xBF80;
    }
    if (tid == 0) cmm::umma::mbar_init(bar, 1);
    cmm::umma::fence_async_smem();
    cmm::tm::fence_before();
    __syncthreads();
    cmm::tm::fence_after();
    const uint32_t ta = s_taddr;
    const uint32_t lane_addr = ta + ((uint32_t)(32 * (warp & 3)) << 16);
    const int cq = warp >> 2;   // this warp's quarter of the columns
    // H as the A operand: TMEM lane i, column c = (H[i][2c], H[i][2c + 1])
    {
        const int i = 32 * (warp & 3) + lane;
        uint32_t w[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int c = 16 * cq + e;
            w[e] = bf16x2((float)hsign(i, 2 * c), (float)hsign(i, 2 * c + 1));
        }
        cmm::tm::st16(lane_addr + 16 * cq, w);
        cmm::tm::wait_st();
    }
    const uint32_t idesc = cmm::umma::idesc_f16(false, 128, 128);
    const uint32_t xs = cmm::umma::smem_u32(xop), hs = cmm::umma::smem_u32(hop);
    uint32_t phase = 0;
    int bad = 0;
    long long c0 = clock64();
    for (int it = 0; it < iters; ++it) {
        if (mode == 2 || it == 0) {
            // integer slice -> BF16 operand X (element (n, k) = x[128 k + n]), slice cleared
            for (int j = tid; j < 2048; j += kThreads) {
                const int kc = j >> 7, n = j & 127;
                int4 *src = reinterpret_cast<int4 *>(slice + ((kc * 128 + n) << 3));
                const int4 a = src[0], b = src[1];
                if (mode == 2) {
                    src[0] = make_int4(0, 0, 0, 0);
                    src[1] = make_int4(0, 0, 0, 0);
                }
                uint4 o;
                o.x = bf16x2(int22_to_f(a.x), int22_to_f(a.y));
                o.y = bf16x2(int22_to_f(a.z), int22_to_f(a.w));
                o.z = bf16x2(int22_to_f(b.x), int22_to_f(b.y));
                o.w = bf16x2(int22_to_f(b.z), int22_to_f(b.w));
                *reinterpret_cast<uint4 *>(xop + op_off(n, 8 * kc)) = o;
            }
            cmm::umma::fence_async_smem();
        }
        cmm::tm::fence_before();
        __syncthreads();
        cmm::tm::fence_after();
        if (tid == 0) {
#pragma unroll 1
            for (int kb = 0; kb < 8; ++kb)
                cmm::umma::mma_ts(ta + 64, ta + 8 * kb,
                                  cmm::umma::smem_desc(xs + kb * 4096, 2048, 128), idesc, kb > 0);
            cmm::umma::commit(bar);
        }
        if (!cmm::umma::mbar_wait(bar, phase & 1, kWaitPolls)) bad = 1;
        ++phase;
        cmm::tm::fence_after();
        if (mode != 0 || it == 0) {
            // D1 (FP32) -> BF16 pairs, the A operand of the second product
            uint32_t r0[16], r1[16], w[16];
            cmm::tm::ld16(lane_addr + 64 + 32 * cq, r0);
            cmm::tm::ld16(lane_addr + 64 + 32 * cq + 16, r1);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                w[e] = bf16x2(__uint_as_float(r0[2 * e]), __uint_as_float(r0[2 * e + 1]));
                w[8 + e] = bf16x2(__uint_as_float(r1[2 * e]), __uint_as_float(r1[2 * e + 1]));
            }
            cmm::tm::st16(lane_addr + 192 + 16 * cq, w);
            cmm::tm::wait_st();
        }
        cmm::tm::fence_before();
        __syncthreads();
        cmm::tm::fence_after();
        if (tid == 0) {
#pragma unroll 1
            for (int kb = 0; kb < 8; ++kb)
                cmm::umma::mma_ts(ta + 64, ta + 192 + 8 * kb,
                                  cmm::umma::smem_desc(hs + kb * 4096, 2048, 128), idesc, kb > 0);
            cmm::umma::commit(bar);
        }
        if (!cmm::umma::mbar_wait(bar, phase & 1, kWaitPolls)) bad = 1;
        ++phase;
        cmm::tm::fence_after();
    }
    const long long c1 = clock64();
    if (bad) {
        atomicOr(status, 1);
        // give the products in flight a second bounded wait before TMEM is freed
        cmm::umma::mbar_wait(bar, (phase - 1) & 1, kWaitPolls);
    }
    if (tid == 0) atomicAdd(&g_clk, (unsigned long long)(c1 - c0));
    if (blockIdx.x == 0 && yout != nullptr) {
        uint32_t r[16];
        const int i = 32 * (warp & 3) + lane;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            cmm::tm::ld16(lane_addr + 64 + 32 * cq + 16 * h, r);
#pragma unroll
            for (int e = 0; e < 16; ++e) yout[i * 128 + 32 * cq + 16 * h + e] = __uint_as_float(r[e]);
        }
    }
    cmm::tm::fence_before();
    __syncthreads();
    cmm::tm::fence_after();
    if (warp == 0) cmm::tm::dealloc(ta, kCols);
}

int hsign_host(int i, int k) {
    int c = 0;
    for (int v = i & k; v; v &= v - 1) ++c;
    return (c & 1) ? -1 : 1;
}

}  // namespace

int main(int argc, char **argv) {
    const int iters = argc > 1 ? std::atoi(argv[1]) : 2000;
    int dev = 0, sms = 0, clk_khz = 0;
    CHECK(cudaGetDevice(&dev));
    CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CHECK(cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev));
    CHECK(cudaFuncSetAttribute(umma_hadamard, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
    // the check: Y = H X H of a {-1, 0, 1} slice, exact
    std::vector<int8_t> x(128 * 128);
    uint32_t s = 12345u;
    for (auto &v : x) {
        s = s * 1664525u + 1013904223u;
        v = (int8_t)((int)(s >> 30) % 3 - 1);
    }
    std::vector<long long> d1(128 * 128, 0);
    std::vector<float> ref(128 * 128);
    for (int i = 0; i < 128; ++i)
        for (int n = 0; n < 128; ++n) {
            long long a = 0;
            for (int k = 0; k < 128; ++k) a += hsign_host(i, k) * x[128 * k + n];
            d1[128 * i + n] = a;
        }
    for (int i = 0; i < 128; ++i)
        for (int j = 0; j < 128; ++j) {
            long long a = 0;
            for (int n = 0; n < 128; ++n) a += d1[128 * i + n] * hsign_host(n, j);
            ref[128 * i + j] = (float)a;
        }
    int8_t *dx = nullptr;
    float *dy = nullptr;
    int *dst = nullptr;
    CHECK(cudaMalloc(&dx, x.size()));
    CHECK(cudaMalloc(&dy, sizeof(float) * 128 * 128));
    CHECK(cudaMalloc(&dst, sizeof(int)));
    CHECK(cudaMemcpy(dx, x.data(), x.size(), cudaMemcpyHostToDevice));
    std::printf("{\"sms\": %d, \"iters\": %d", sms, iters);
    int rc = 0;
    for (int mode = 0; mode < 3; ++mode) {
        // correctness (one slice), then timing (iters slices per CTA, one CTA per SM)
        CHECK(cudaMemset(dst, 0, sizeof(int)));
        CHECK(cudaMemset(dy, 0, sizeof(float) * 128 * 128));
        umma_hadamard<<<1, kThreads, kSmem>>>(mode, 1, dx, dy, dst);
        CHECK(cudaDeviceSynchronize());
        std::vector<float> y(128 * 128);
        int st = 0;
        CHECK(cudaMemcpy(y.data(), dy, sizeof(float) * y.size(), cudaMemcpyDeviceToHost));
        CHECK(cudaMemcpy(&st, dst, sizeof(int), cudaMemcpyDeviceToHost));
        int wrong = 0;
        for (size_t e = 0; e < y.size(); ++e) wrong += y[e] != ref[e];
        const unsigned long long zero = 0;
        CHECK(cudaMemcpyToSymbol(g_clk, &zero, sizeof zero));
        cudaEvent_t e0, e1;
        CHECK(cudaEventCreate(&e0));
        CHECK(cudaEventCreate(&e1));
        umma_hadamard<<<sms, kThreads, kSmem>>>(mode, 16, dx, nullptr, dst);   // warm-up
        CHECK(cudaMemcpyToSymbol(g_clk, &zero, sizeof zero));
        CHECK(cudaEventRecord(e0));
        umma_hadamard<<<sms, kThreads, kSmem>>>(mode, iters, dx, nullptr, dst);
        CHECK(cudaEventRecord(e1));
        CHECK(cudaEventSynchronize(e1));
        CHECK(cudaGetLastError());
        float ms = 0.f;
        CHECK(cudaEventElapsedTime(&ms, e0, e1));
        unsigned long long clk = 0;
        CHECK(cudaMemcpyFromSymbol(&clk, g_clk, sizeof clk));
        CHECK(cudaMemcpy(&st, dst, sizeof(int), cudaMemcpyDeviceToHost));
        const double clk_per_slice = (double)clk / sms / iters;
        const double flops = 4.0 * 128.0 * 128.0 * 128.0 * (double)sms * iters;
        std::printf(", \"mode%d\": {\"wrong\": %d, \"status\": %d, \"ms\": %.4f, "
                    "\"clk_per_slice_per_sm\": %.1f, \"tflops\": %.1f}",
                    mode, wrong, st, ms, clk_per_slice, flops / (ms * 1e-3) / 1e12);
        if (wrong || st) rc = 2;
        CHECK(cudaEventDestroy(e0));
        CHECK(cudaEventDestroy(e1));
    }
    std::printf(", \"clock_khz_attr\": %d}\n", clk_khz);
    CHECK(cudaFree(dx));
    CHECK(cudaFree(dy));
    CHECK(cudaFree(dst));
    return rc;
}
