// alu_rates.cu -- throughput of the arithmetic the sketch kernels are built
// from, measured on the device it runs on: FP32 add (scalar and packed
// FP32x2), FP64 add, 32- and 64-bit integer add, 64-bit integer radix-4
// butterflies, 32-bit integer multiply-add,
// 64-bit -> FP32 and 32-bit -> FP32 conversions, and 32- / 64-bit integer
// atomic adds to distinct shared-memory words.  Each kernel runs a fixed
// number of independent operation chains per thread (no memory traffic in
// the loop); the result is operations per clock per SM and per second.
// Built and run by probes/run_alu_rates.py; it writes one JSON line.
//
// Bounds: every kernel writes exactly one word per thread to `sink`, which
// holds gridDim.x * blockDim.x words; shared-memory indices are threadIdx.x
// (+ a multiple of 32 below the 4096-word array).
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define CHECK(x)                                                                     \
    do {                                                                             \
        cudaError_t e_ = (x);                                                        \
        if (e_ != cudaSuccess) {                                                     \
            std::fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));            \
            return 1;                                                                \
        }                                                                            \
    } while (0)

constexpr int kThreads = 256;
constexpr int kChains = 8;     // independent chains per thread
constexpr int kIters = 4096;   // loop trips; each trip = kChains operations

__device__ unsigned long long g_clk_sum;   // summed clock64 deltas of the first warp of each CTA

__device__ __forceinline__ void note_clock(long long c0) {
    if (threadIdx.x == 0) atomicAdd(&g_clk_sum, (unsigned long long)(clock64() - c0));
}

__global__ void k_fadd(float *sink, float y) {
    const long long c0 = clock64();
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3f + c;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = x[c] + y;
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
    note_clock(c0);
}

// packed FP32x2: one instruction adds two lanes' pairs (counted as 2 ops)
__global__ void k_fadd2(float *sink, float y) {
    const long long c0 = clock64();
    float2 x[kChains / 2];
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) x[c] = make_float2(threadIdx.x * 1e-3f + c, c);
    const float2 y2 = make_float2(y, y);
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains / 2; ++c) x[c] = __fadd2_rn(x[c], y2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) s += x[c].x + x[c].y;
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
    note_clock(c0);
}

__global__ void k_dadd(float *sink, double y) {
    const long long c0 = clock64();
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3 + c;
    for (int it = 0; it < kIters / 16; ++it) {   // FP64 is slow: fewer trips (scaled on the host)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = x[c] + y;
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
    note_clock(c0);
}

// integer ops through inline PTX so that the compiler cannot fold the chains
__global__ void k_iadd32(float *sink, int y) {
    const long long c0 = clock64();
    int x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x + c;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm volatile("add.s32 %0, %0, %1;" : "+r"(x[c]) : "r"(y));
    }
    int s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= x[c];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
    note_clock(c0);
}

__global__ void k_iadd64(float *sink, long long y) {
    const long long c0 = clock64();
    long long x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x + c;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm volatile("add.s64 %0, %0, %1;" : "+l"(x[c]) : "l"(y));
    }
    long long s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= x[c];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
    note_clock(c0);
}

__global__ void k_imad32(float *sink, int y) {
    const long long c0 = clock64();
    int x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x + c;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm volatile("mad.lo.s32 %0, %0, %1, %1;" : "+r"(x[c]) : "r"(y));
    }
    int s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= x[c];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
    note_clock(c0);
}

// conversions: each trip converts kChains independent integers and adds the
// results into kChains float accumulators (the adds are counted separately
// by k_fadd; the conversion rate is the lower one)
__global__ void k_cvt_s64_f32(float *sink, long long y) {
    const long long c0 = clock64();
    long long v[kChains];
    float acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        v[c] = (long long)threadIdx.x * 977 + c;
        acc[c] = 0.f;
    }
    for (int it = 0; it < kIters / 4; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float f;
            asm volatile("cvt.rn.f32.s64 %0, %1;" : "=f"(f) : "l"(v[c] + it * y));
            acc[c] += f;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
    note_clock(c0);
}

__global__ void k_cvt_s32_f32(float *sink, int y) {
    const long long c0 = clock64();
    int v[kChains];
    float acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        v[c] = threadIdx.x * 977 + c;
        acc[c] = 0.f;
    }
    for (int it = 0; it < kIters / 4; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float f;
            asm volatile("cvt.rn.f32.s32 %0, %1;" : "=f"(f) : "r"(v[c] + it * y));
            acc[c] += f;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
    note_clock(c0);
}

// shared-memory integer atomics, 32 lanes on 32 distinct banks (word = lane +
// 32 * chain for 32-bit; for 64-bit, lanes 2 words apart, a half-warp per
// 128-byte row)
__global__ void k_atoms32(float *sink, int y) {
    __shared__ int sm[4096];
    const long long c0 = clock64();
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) sm[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;   // 8 warps
    for (int it = 0; it < kIters / 8; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) atomicAdd(&sm[lane + 32 * ((w * kChains + c) & 127)], y);
    }
    __syncthreads();
    sink[blockIdx.x * blockDim.x + threadIdx.x] = (float)sm[threadIdx.x];
    note_clock(c0);
}

__global__ void k_atoms64(float *sink, unsigned long long y) {
    __shared__ unsigned long long sm[2048];
    const long long c0 = clock64();
    for (int i = threadIdx.x; i < 2048; i += blockDim.x) sm[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int it = 0; it < kIters / 8; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) atomicAdd(&sm[lane + 32 * ((w * kChains + c) & 63)], y);
    }
    __syncthreads();
    sink[blockIdx.x * blockDim.x + threadIdx.x] = (float)sm[threadIdx.x];
    note_clock(c0);
}

// Walsh-Hadamard butterflies on 64-bit integers in the form the fixed-point
// sketch runs them: 16 values per thread, four stages as two radix-4 passes
// (each output one three-input add or subtract), counted as one operation per
// value per stage.  A constant added to one value per transform keeps the
// values from settling; 64 registers at most, so that 4 CTAs stay resident.
__global__ void __launch_bounds__(kThreads, 4) k_r4_s64(float *sink, long long y) {
    const long long c0 = clock64();
    long long v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = threadIdx.x * 16 + j;
    for (int it = 0; it < kIters / 8; ++it) {
#pragma unroll
        for (int h = 1; h < 16; h *= 4) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                if ((j & (3 * h)) == 0) {
                    const long long a = v[j], b = v[j + h], c = v[j + 2 * h], d = v[j + 3 * h];
                    const long long s1 = a + b, d1 = a - b;
                    v[j] = s1 + c + d;
                    v[j + h] = d1 + c - d;
                    v[j + 2 * h] = s1 - c - d;
                    v[j + 3 * h] = d1 - c + d;
                }
            }
        }
        v[0] += y;
    }
    long long s = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) s ^= v[j];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
    note_clock(c0);
}

template <typename K, typename Y>
int run(const char *name, K kern, Y y, double ops_per_thread, int sms, float *sink, int blocks,
        bool first) {
    cudaEvent_t e0, e1;
    CHECK(cudaEventCreate(&e0));
    CHECK(cudaEventCreate(&e1));
    kern<<<blocks, kThreads>>>(sink, y);   // warm-up
    CHECK(cudaGetLastError());
    CHECK(cudaDeviceSynchronize());
    unsigned long long zero = 0;
    CHECK(cudaMemcpyToSymbol(g_clk_sum, &zero, sizeof zero));
    CHECK(cudaEventRecord(e0));
    kern<<<blocks, kThreads>>>(sink, y);
    CHECK(cudaEventRecord(e1));
    CHECK(cudaEventSynchronize(e1));
    CHECK(cudaGetLastError());
    float ms = 0.f;
    CHECK(cudaEventElapsedTime(&ms, e0, e1));
    unsigned long long clk = 0;
    CHECK(cudaMemcpyFromSymbol(&clk, g_clk_sum, sizeof clk));
    const double total_ops = ops_per_thread * (double)blocks * kThreads;
    const double per_s = total_ops / (ms * 1e-3);
    // clocks: CTAs run in waves of `resident` per SM; each CTA's clock span is
    // about the time of its wave, so the mean span times the number of waves
    // is the SM-clock count of the kernel
    const double mean_span = (double)clk / blocks;
    const int per_sm = blocks / sms;
    const double sm_clocks = mean_span;   // one wave: all CTAs resident at once
    const double per_clk_sm = total_ops / sms / sm_clocks;
    const double mhz = sm_clocks / (ms * 1e-3) / 1e6;
    std::printf("%s\"%s\": {\"ms\": %.4f, \"ops_per_s\": %.4e, \"ops_per_clk_per_sm\": %.2f, "
                "\"sm_mhz_in_kernel\": %.0f, \"ctas_per_sm\": %d}",
                first ? "" : ", ", name, ms, per_s, per_clk_sm, mhz, per_sm);
    CHECK(cudaEventDestroy(e0));
    CHECK(cudaEventDestroy(e1));
    return 0;
}

int main() {
    int dev = 0, sms = 0;
    CHECK(cudaGetDevice(&dev));
    CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // 4 CTAs of 256 threads per SM, all resident at once (one wave)
    const int blocks = sms * 4;
    float *sink = nullptr;
    CHECK(cudaMalloc(&sink, sizeof(float) * blocks * kThreads));
    const double n = (double)kIters * kChains;
    std::printf("{\"sms\": %d, ", sms);
    int rc = 0;
    rc |= run("fadd_f32", k_fadd, 1.0f, n, sms, sink, blocks, true);
    rc |= run("fadd2_f32x2", k_fadd2, 1.0f, n, sms, sink, blocks, false);
    rc |= run("dadd_f64", k_dadd, 1.0, n / 16, sms, sink, blocks, false);
    rc |= run("add_s32", k_iadd32, 3, n, sms, sink, blocks, false);
    rc |= run("add_s64", k_iadd64, 3ll, n, sms, sink, blocks, false);
    rc |= run("fwht_r4_s64", k_r4_s64, 3ll, (double)(kIters / 8) * 4 * 16, sms, sink, blocks, false);
    rc |= run("mad_lo_s32", k_imad32, 3, n, sms, sink, blocks, false);
    rc |= run("cvt_f32_s64", k_cvt_s64_f32, 3ll, n / 4, sms, sink, blocks, false);
    rc |= run("cvt_f32_s32", k_cvt_s32_f32, 3, n / 4, sms, sink, blocks, false);
    rc |= run("atom_shared_add_u32", k_atoms32, 1, n / 8, sms, sink, blocks, false);
    rc |= run("atom_shared_add_u64", k_atoms64, 1ull, n / 8, sms, sink, blocks, false);
    std::printf("}\n");
    CHECK(cudaFree(sink));
    return rc;
}
