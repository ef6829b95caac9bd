// layout_check.cu -- host-only check of the shared-memory index maps the
// register-round transforms use (fwht_device.cuh), for every instantiation the
// kernels launch.  Built and run by tests/test_layouts_host.py; no GPU needed:
// only the constexpr __host__ __device__ index functions are called.
//
// For each (T, L, LE, threads) and each register round K it checks that
//  - (thread q, register j) -> u covers [0, 2^L) exactly once (a bijection),
//  - the padded word of u is injective and below the group's stride,
//  - the accesses are free of shared-memory bank conflicts: per warp for
//    32-bit words, per half-warp for 64-bit words, and per quarter-warp of
//    16-byte chunks (16-byte aligned, contiguous) for the vectorised FP32 round 0.
// Prints one line per failure and exits non-zero if any.
#include <cstdio>
#include <vector>

#include "fwht_device.cuh"

using namespace cmm;

static int g_fail = 0;

template <typename T, int L, int LE, int K>
static void check_round(int threads) {
    using S = FwhtShape<T, L, LE>;
    using RK = typename S::template Round<K>;
    constexpr int N = S::N, E = S::E, P = S::P;
    const int G = threads / P;
    const char *tn = sizeof(T) == 4 ? "f32" : "64-bit";
    if (G < 1 || threads % P != 0) {
        std::printf("%s L=%d LE=%d threads=%d: groups do not tile the CTA\n", tn, L, LE, threads);
        ++g_fail;
        return;
    }
    std::vector<int> seen(N, 0), used(S::STRIDE, 0);
    for (int q = 0; q < P; ++q)
        for (int j = 0; j < E; ++j) {
            const int u = RK::u(q, j);
            if (u < 0 || u >= N || seen[u]++) {
                std::printf("%s L=%d LE=%d K=%d: u(%d,%d)=%d repeats or is out of range\n", tn, L,
                            LE, K, q, j, u);
                ++g_fail;
                return;
            }
            const int w = RK::addr(q, j);
            if (w < 0 || w >= S::STRIDE || used[w]++) {
                std::printf("%s L=%d LE=%d K=%d: word %d repeats or is out of range\n", tn, L, LE,
                            K, w);
                ++g_fail;
                return;
            }
        }
    const bool vec = K == 0 && sizeof(T) == 4 && S::PAD == 4;
    auto word = [&](int tid, int j) { return (tid / P) * S::STRIDE + RK::addr(tid % P, j); };
    for (int w0 = 0; w0 < threads; w0 += 32) {
        if (vec) {
            // 16-byte chunks: each row contiguous and aligned; per quarter-warp
            // the 8 chunks fall in 8 distinct groups of 4 banks
            for (int c = 0; c < E / 4; ++c)
                for (int qw = 0; qw < 4; ++qw) {
                    int grp[8], n = 0;
                    for (int l = 0; l < 8; ++l) {
                        const int tid = w0 + 8 * qw + l;
                        if (tid >= threads) continue;
                        const int a = word(tid, 4 * c);
                        for (int e = 1; e < 4; ++e)
                            if (word(tid, 4 * c + e) != a + e) {
                                std::printf("f32 L=%d LE=%d: row not contiguous\n", L, LE);
                                ++g_fail;
                                return;
                            }
                        if (a % 4) {
                            std::printf("f32 L=%d LE=%d: row not 16-byte aligned\n", L, LE);
                            ++g_fail;
                            return;
                        }
                        grp[n++] = (a / 4) % 8;
                    }
                    for (int x = 0; x < n; ++x)
                        for (int y = x + 1; y < n; ++y)
                            if (grp[x] == grp[y]) {
                                std::printf("f32 L=%d LE=%d K=0: vector bank conflict\n", L, LE);
                                ++g_fail;
                                return;
                            }
                }
            continue;
        }
        const int span = sizeof(T) == 4 ? 32 : 16;   // lanes served per wavefront
        for (int j = 0; j < E; ++j)
            for (int h = 0; h < 32; h += span) {
                int bank_word[32];
                for (int b = 0; b < 32; ++b) bank_word[b] = -1;
                for (int l = 0; l < span; ++l) {
                    const int tid = w0 + h + l;
                    if (tid >= threads) continue;
                    const int wd = word(tid, j);
                    for (int half = 0; half < (int)(sizeof(T) / 4); ++half) {
                        const int b = (wd * (int)(sizeof(T) / 4) + half) % 32;
                        const int id = wd * 2 + half;
                        if (bank_word[b] != -1 && bank_word[b] != id) {
                            std::printf("%s L=%d LE=%d K=%d threads=%d: bank conflict (j=%d)\n", tn,
                                        L, LE, K, threads, j);
                            ++g_fail;
                            return;
                        }
                        bank_word[b] = id;
                    }
                }
            }
    }
}

template <typename T, int L, int LE, int K>
static void check_rounds(int threads) {
    if constexpr (K < FwhtShape<T, L, LE>::NR) {
        check_round<T, L, LE, K>(threads);
        check_rounds<T, L, LE, K + 1>(threads);
    }
}

template <typename T, int L, int LE>
static void check(int threads) {
    check_rounds<T, L, LE, 0>(threads);
}

template <int L>
static void all_l() {
    constexpr int LE32 = L < 5 ? L : 5, LE64 = L < 4 ? L : 4;
    // single-problem sketch kernels
    check<float, L, LE32>(L == 14 ? 512 : 256);
    if constexpr (L <= 13) check<double, L, LE64>(L == 13 ? 512 : 256);
    // exact fixed-point (int64) sketch kernel: 256 threads, 32 values per thread
    if constexpr (L <= 13) check<long long, L, LE32>(256);
    // batched sketch tasks: 512 threads, slices 2^5 .. 2^14
    if constexpr (L >= 5) check<float, L, 5>(512);
    // adjoint kernel: max(P, 256) threads
    constexpr int P32 = (1 << L) >> LE32, P64 = (1 << L) >> LE64;
    check<float, L, LE32>(P32 >= 256 ? P32 : 256);
    if constexpr (L <= 13) check<double, L, LE64>(P64 >= 256 ? P64 : 256);
}

template <int... Ls>
static void all(std::integer_sequence<int, Ls...>) {
    (all_l<Ls + 1>(), ...);
}

int main() {
    all(std::make_integer_sequence<int, 14>{});
    if (g_fail) {
        std::printf("%d layout checks failed\n", g_fail);
        return 1;
    }
    std::printf("layout checks passed\n");
    return 0;
}
