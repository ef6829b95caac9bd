// umma_desc_check.cu -- host-only check of the tensor-core descriptor
// encodings in umma_device.cuh: each field decoded back out of the 64-bit
// shared-memory descriptor and the 32-bit instruction descriptor equals the
// value put in, the reserved bits stay zero.  Built and run by
// tests/test_gpu_umma_probe.py; no GPU needed.
#include <cstdint>
#include <cstdio>

#include "umma_device.cuh"

using namespace cmm;

static int g_fail = 0;

static void expect(const char *what, uint64_t got, uint64_t want) {
    if (got != want) {
        std::printf("%s: %llu, expected %llu\n", what, (unsigned long long)got,
                    (unsigned long long)want);
        ++g_fail;
    }
}

int main() {
    const uint32_t addrs[] = {0u, 16u, 0x1000u, 0x10000u, 0x38FF0u};
    const uint32_t offs[] = {16u, 128u, 2048u, 4096u, 0x3FFF0u};
    for (uint32_t a : addrs)
        for (uint32_t l : offs)
            for (uint32_t s : offs) {
                const uint64_t d = umma::smem_desc(a, l, s);
                expect("start", d & 0x3FFF, a >> 4);
                expect("leading offset", (d >> 16) & 0x3FFF, l >> 4);
                expect("stride offset", (d >> 32) & 0x3FFF, s >> 4);
                expect("version", (d >> 46) & 0x7, 1);
                expect("base offset, mode, reserved", (d >> 49) & 0xFFF, 0);
                expect("swizzle", d >> 61, 0);
                expect("reserved 14-15, 30-31", d & 0xC000C000ull, 0);
            }
    for (int f16 = 0; f16 < 2; ++f16)
        for (int M : {64, 128, 256})
            for (int N = 16; N <= 256; N += 16) {
                const uint32_t i = umma::idesc_f16(f16 != 0, M, N);
                expect("sparsity, saturate", i & 0xF, 0);
                expect("D format F32", (i >> 4) & 3, 1);
                expect("A format", (i >> 7) & 7, f16 ? 0 : 1);
                expect("B format", (i >> 10) & 7, f16 ? 0 : 1);
                expect("negate, major", (i >> 13) & 0xF, 0);
                expect("N >> 3", (i >> 17) & 0x3F, (uint64_t)(N >> 3));
                expect("M >> 4", (i >> 24) & 0x1F, (uint64_t)(M >> 4));
                expect("reserved 6, 23, 29-31", i & 0xE0800040u, 0);
            }
    if (g_fail) return 1;
    std::printf("descriptor checks passed\n");
    return 0;
}
