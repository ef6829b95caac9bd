// umma_device.cuh -- the fifth-generation tensor-core operations (tcgen05.mma)
// the Hadamard-block sketch kernel issues: shared-memory matrix descriptors,
// instruction descriptors for 16-bit operands with FP32 accumulation, the
// asynchronous products (A from shared or tensor memory, B from shared
// memory, D in tensor memory), their completion through an mbarrier, and the
// bounded waits on it.
//
// Shared-memory operands use the K-major layout without swizzling: the
// matrix is cut into core matrices of 8 rows x 16 bytes (8 x 8 16-bit
// values), each stored as 128 contiguous bytes (row r of the core matrix at
// byte 16 r); the descriptor gives the byte distance between core matrices
// adjacent along K (leading-dimension offset) and along M or N (stride-
// dimension offset).
#pragma once

#include <cstdint>

namespace cmm {
namespace umma {

// shared-memory matrix descriptor: start address, leading- and stride-
// dimension byte offsets (all multiples of 16 bytes, encoded >> 4), the
// descriptor version 1 of this architecture (bits 46-48 = 0b001), base
// offset 0, no swizzling (bits 61-63 = 0)
__host__ __device__ constexpr uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D in FP32 (bits 4-5 = 1), A and B
// both BF16 (bits 7-9 and 10-12 = 1) or both FP16 (0), no negation, both
// K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28
__host__ __device__ constexpr uint32_t idesc_f16(bool f16, int M, int N) {
    return (1u << 4) | ((f16 ? 0u : 1u) << 7) | ((f16 ? 0u : 1u) << 10) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// D (tensor memory) = A (tensor memory) . B (shared memory) [+ D when acc]
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                       uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
        :
        : "r"(d_tmem), "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(acc)
        : "memory");
}

// D (tensor memory) = A (shared memory) . B (shared memory) [+ D when acc]
__device__ __forceinline__ void mma_ss(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                       uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :
        : "r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(acc)
        : "memory");
}

// the mbarrier at `bar` receives one arrival when every tcgen05 operation
// this thread issued before has completed
__device__ __forceinline__ void commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// wait for phase `parity` of the mbarrier to complete, at most `limit` polls
// (each try_wait itself suspends for a bounded time); false when it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try(bar, parity)) return true;
    return false;
}

// generic-proxy writes to shared memory made visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace umma
}  // namespace cmm
