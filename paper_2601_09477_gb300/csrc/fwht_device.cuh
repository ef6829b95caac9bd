// fwht_device.cuh -- in-CTA Walsh-Hadamard transform of a shared-memory slice.
//
// A "group" of P threads transforms one slice of N = 2^L values held in shared
// memory.  Each thread keeps E = 2^LE values in registers; the L butterfly
// stages (H[u][v] = (-1)^popcount(u & v), Sylvester order, unnormalised) are
// done in ceil(L / LE) register rounds, round K covering index bits
// [K*LE, K*LE + nb_K).  Between rounds the slice goes through shared memory.
//
// Layout: element u lives at word u + (u >> LE) of the group's array (one pad
// word per E words).  With that padding every round's loads and stores are free
// of bank conflicts for 4-byte elements (and per half-warp for 8-byte ones),
// and the address of (thread q, register j) splits into a per-thread base plus
// a compile-time offset, so the compiler uses [reg + imm] addressing.
#pragma once

#include <cstdint>

namespace cmm {

template <int LE>
__host__ __device__ constexpr int pad_index(int u) { return u + (u >> LE); }

template <int L, int LE>
struct FwhtShape {
    static constexpr int N = 1 << L;
    static constexpr int E = 1 << LE;
    static constexpr int P = N / E;                  // threads per group
    static constexpr int NR = (L + LE - 1) / LE;     // register rounds
    static constexpr int STRIDE = N + N / E;         // words per group array (with pads)
    static_assert(LE <= L, "register block larger than the transform");

    template <int K>
    struct Round {
        static constexpr int lo = K * LE;
        static constexpr int nb = (L - lo) < LE ? (L - lo) : LE;
        // index u of register j of thread q: the low nb bits of j are the
        // transformed bits [lo, lo+nb); the remaining register bits, then the
        // thread bits, fill the other index bits from the bottom up.
        __host__ __device__ static constexpr int u(int q, int j) {
            int payload = (j >> nb) | (q << (LE - nb));
            int low = payload & ((1 << lo) - 1);
            int high = payload >> lo;
            return low | ((j & ((1 << nb) - 1)) << lo) | (high << (lo + nb));
        }
        __host__ __device__ static constexpr int addr(int q, int j) {
            return pad_index<LE>(u(q, j));
        }
    };
};

// butterflies over the low NB bits of the register index, independently for
// every value of the remaining register bits
template <typename T, int E, int NB>
__device__ __forceinline__ void reg_fwht(T (&v)[E]) {
#pragma unroll
    for (int s = 0; s < NB; ++s) {
#pragma unroll
        for (int j = 0; j < E; ++j) {
            if (!(j & (1 << s))) {
                const T a = v[j];
                const T b = v[j | (1 << s)];
                v[j] = a + b;
                v[j | (1 << s)] = a - b;
            }
        }
    }
}

// barrier of one group: named barrier for multi-warp groups, warp barrier for
// groups of at most one warp (all lanes of a warp run the same trip counts)
template <int P>
__device__ __forceinline__ void group_sync(int g) {
    if constexpr (P >= 64) {
        asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(P) : "memory");
    } else {
        __syncwarp();
    }
}

// Transform the group's slice Sg in place, leaving the result in registers v
// (round NR-1 layout) and the shared array zeroed for the next scatter.
template <typename T, int L, int LE, int K>
__device__ __forceinline__ void fwht_rounds(T *Sg, T (&v)[1 << LE], int q, int g) {
    using S = FwhtShape<L, LE>;
    using RK = typename S::template Round<K>;
    constexpr int E = S::E;
    T *base = Sg + RK::addr(q, 0);
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = base[RK::addr(0, j)];
    reg_fwht<T, E, RK::nb>(v);
    if constexpr (K + 1 < S::NR) {
#pragma unroll
        for (int j = 0; j < E; ++j) base[RK::addr(0, j)] = v[j];
        group_sync<S::P>(g);
        fwht_rounds<T, L, LE, K + 1>(Sg, v, q, g);
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j) base[RK::addr(0, j)] = T(0);
    }
}

// index (in the unpadded slice) of register j of thread q after the last round
template <int L, int LE>
__device__ __forceinline__ int final_index(int q, int j) {
    using S = FwhtShape<L, LE>;
    return S::template Round<S::NR - 1>::u(q, j);
}

// top bits of (a x + c) mod 2^64: the multiply-add-shift hash of Sec. 4.2
__device__ __forceinline__ uint32_t mas_hash(uint64_t a, uint64_t c, uint64_t x, int shift) {
    return (uint32_t)((a * x + c) >> shift);
}

__device__ __forceinline__ uint32_t mas_sign_bit(uint64_t a, uint64_t c, uint64_t x) {
    return (uint32_t)((a * x + c) >> 63);   // 1 means the sign -1
}

}  // namespace cmm
