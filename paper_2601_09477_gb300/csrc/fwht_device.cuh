// fwht_device.cuh -- in-CTA Walsh-Hadamard transform of a shared-memory slice.
//
// A "group" of P threads transforms one slice of N = 2^L values held in shared
// memory.  Each thread keeps E = 2^LE values in registers; the L butterfly
// stages (H[u][v] = (-1)^popcount(u & v), Sylvester order, unnormalised) are
// done in ceil(L / LE) register rounds, round K covering index bits
// [K*LE, K*LE + nb_K).  Between rounds the slice goes through shared memory.
//
// Layout: element u lives at word u + PAD * (u >> LE) of the group's array.
// For FP32 with E = 32 and N >= 2^10, PAD = 4: each 32-element row of round 0
// is contiguous and 16-byte aligned (vector loads and stores), and the loads
// and stores of every round are free of bank conflicts (the thread index fills
// the low complement bits, so the 32 lanes of a warp hit 32 distinct banks).
// Smaller FP32 transforms (several groups per warp) and FP64 use PAD = 1,
// which is conflict-free for them (per half-warp for FP64).  The address of (thread q,
// register j) splits into a per-thread base plus a compile-time offset.
//
// FP32 butterflies of stages >= 1 run as packed FP32x2 operations (two
// independent IEEE additions per instruction, identical results to scalar
// adds); a - b is formed as fma(b, -1, a), which is exact-rounded a - b.
#pragma once

#include <cstdint>

namespace cmm {

template <typename T, int L, int LE>
struct PadOf {
    // 4 pad words per 32-word row for FP32 transforms of 2^10 and more (vector
    // rows in round 0); 1 otherwise (several groups share a warp below 2^10)
    static constexpr int value = (sizeof(T) == 4 && LE >= 5 && L >= 10) ? 4 : 1;
};

template <typename T, int L, int LE>
__host__ __device__ constexpr int pad_index(int u) {
    return u + PadOf<T, L, LE>::value * (u >> LE);
}

template <typename T, int L, int LE>
struct FwhtShape {
    static constexpr int N = 1 << L;
    static constexpr int E = 1 << LE;
    static constexpr int P = N / E;                  // threads per group
    static constexpr int NR = (L + LE - 1) / LE;     // register rounds
    static constexpr int PAD = PadOf<T, L, LE>::value;
    static constexpr int STRIDE = N + PAD * (N / E); // words per group array (with pads)
    static_assert(LE <= L, "register block larger than the transform");

    template <int K>
    struct Round {
        static constexpr int lo = K * LE;
        static constexpr int nb = (L - lo) < LE ? (L - lo) : LE;
        // index u of register j of thread q: the low nb bits of j are the
        // transformed bits [lo, lo+nb); the thread bits fill the other index
        // bits from the bottom up, then the remaining register bits
        __host__ __device__ static constexpr int u(int q, int j) {
            const int payload = q | ((j >> nb) << (L - LE));
            const int low = payload & ((1 << lo) - 1);
            const int high = payload >> lo;
            return low | ((j & ((1 << nb) - 1)) << lo) | (high << (lo + nb));
        }
        __host__ __device__ static constexpr int addr(int q, int j) {
            return pad_index<T, L, LE>(u(q, j));
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

// Butterflies over the low NB bits of the register index, two stages at a
// time where possible: for a, b, c, d at offsets 0, h, 2h, 3h,
//   a' = (a + b) + (c + d)   b' = (a - b) + (c - d)
//   c' = (a + b) - (c + d)   d' = (a - b) - (c - d),
// written as three-operand sums so that each output is one three-input
// integer add (with carries for 64-bit values): 6 adds for 8 butterfly
// outputs instead of 8; an odd last stage is a plain radix-2 stage.  For
// integer T only (exact, or modular for unsigned packed words), where the
// result equals the stage-by-stage transform.
template <typename T, int E, int NB>
__device__ __forceinline__ void reg_fwht_r4(T (&v)[E]) {
#pragma unroll
    for (int s = 0; s + 1 < NB; s += 2) {
        const int h = 1 << s;
#pragma unroll
        for (int j = 0; j < E; ++j) {
            if ((j & (3 * h)) == 0) {
                const T a = v[j], b = v[j + h], c = v[j + 2 * h], d = v[j + 3 * h];
                const T s1 = a + b, d1 = a - b;
                v[j] = s1 + c + d;
                v[j + h] = d1 + c - d;
                v[j + 2 * h] = s1 - c - d;
                v[j + 3 * h] = d1 - c + d;
            }
        }
    }
    if constexpr (NB % 2 == 1) {
        constexpr int h = 1 << (NB - 1);
#pragma unroll
        for (int j = 0; j < E; ++j) {
            if (!(j & h)) {
                const T a = v[j], b = v[j + h];
                v[j] = a + b;
                v[j + h] = a - b;
            }
        }
    }
}

// FP32: stage 0 scalar, stages >= 1 on packed pairs (j, j+1) and (j+h, j+h+1);
// SKIP0 leaves out stage 0 (done by the caller)
template <int E, int NB, bool SKIP0 = false>
__device__ __forceinline__ void reg_fwht_f32(float (&v)[E]) {
    if constexpr (NB >= 1 && !SKIP0) {
#pragma unroll
        for (int j = 0; j < E; j += 2) {
            const float a = v[j], b = v[j + 1];
            v[j] = a + b;
            v[j + 1] = a - b;
        }
    }
    if constexpr (NB >= 2 && E >= 4) {
        const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
        for (int s = 1; s < NB; ++s) {
#pragma unroll
            for (int j = 0; j < E; j += 2) {
                if (!(j & (1 << s))) {
                    const float2 a = make_float2(v[j], v[j + 1]);
                    const float2 b = make_float2(v[j | (1 << s)], v[(j | (1 << s)) + 1]);
                    const float2 sum = __fadd2_rn(a, b);
                    const float2 dif = __ffma2_rn(b, m1, a);
                    v[j] = sum.x;
                    v[j + 1] = sum.y;
                    v[j | (1 << s)] = dif.x;
                    v[(j | (1 << s)) + 1] = dif.y;
                }
            }
        }
    }
}

template <typename T, int E, int NB>
__device__ __forceinline__ void reg_fwht_any(T (&v)[E]) {
    if constexpr (sizeof(T) == 4) {
        reg_fwht_f32<E, NB>(v);
    } else {
        reg_fwht<T, E, NB>(v);
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

// load / store the E values of round K (vectorised for the contiguous,
// 16-byte aligned rows of FP32 round 0)
template <typename T, int L, int LE, int K>
__device__ __forceinline__ void round_load(const T *base, T (&v)[1 << LE]) {
    using RK = typename FwhtShape<T, L, LE>::template Round<K>;
    constexpr int E = 1 << LE;
    if constexpr (K == 0 && PadOf<T, L, LE>::value == 4) {
        const float4 *b4 = reinterpret_cast<const float4 *>(base);
#pragma unroll
        for (int c = 0; c < E / 4; ++c) {
            const float4 w = b4[c];
            v[4 * c] = w.x;
            v[4 * c + 1] = w.y;
            v[4 * c + 2] = w.z;
            v[4 * c + 3] = w.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j) v[j] = base[RK::addr(0, j)];
    }
}

template <typename T, int L, int LE, int K>
__device__ __forceinline__ void round_store(T *base, const T (&v)[1 << LE]) {
    using RK = typename FwhtShape<T, L, LE>::template Round<K>;
    constexpr int E = 1 << LE;
    if constexpr (K == 0 && PadOf<T, L, LE>::value == 4) {
        float4 *b4 = reinterpret_cast<float4 *>(base);
#pragma unroll
        for (int c = 0; c < E / 4; ++c)
            b4[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j) base[RK::addr(0, j)] = v[j];
    }
}

// round-0 load of FP32 values from integer bucket sums (the fixed-point
// scatter): v = float(sum) * inv, inv a power of two
template <int L, int LE>
__device__ __forceinline__ void round_load_fixed(const float *base, float (&v)[1 << LE],
                                                 float inv) {
    using RK = typename FwhtShape<float, L, LE>::template Round<0>;
    constexpr int E = 1 << LE;
    const int *ib = reinterpret_cast<const int *>(base);
    if constexpr (PadOf<float, L, LE>::value == 4) {
        const int4 *b4 = reinterpret_cast<const int4 *>(ib);
#pragma unroll
        for (int c = 0; c < E / 4; ++c) {
            const int4 w = b4[c];
            v[4 * c] = __int2float_rn(w.x) * inv;
            v[4 * c + 1] = __int2float_rn(w.y) * inv;
            v[4 * c + 2] = __int2float_rn(w.z) * inv;
            v[4 * c + 3] = __int2float_rn(w.w) * inv;
        }
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j) v[j] = __int2float_rn(ib[RK::addr(0, j)]) * inv;
    }
}

// last-round load of 32-bit values that also zeroes them for the next
// scatter: one shared-memory exchange per word costs the pipe about what a
// load does, so the separate clearing pass goes (each word is read by exactly
// one thread in a round, so nothing else reads it after it is zeroed)
template <typename T, int L, int LE, int K>
__device__ __forceinline__ void round_load_clear(T *base, T (&v)[1 << LE]) {
    static_assert(sizeof(T) == 4, "32-bit words only");
    using RK = typename FwhtShape<T, L, LE>::template Round<K>;
    constexpr int E = 1 << LE;
    int *ib = reinterpret_cast<int *>(base);
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = __int_as_float(atomicExch(ib + RK::addr(0, j), 0));
}

// Transform the group's slice Sg in place, leaving the result in registers v
// (round NR-1 layout) and the shared array zeroed for the next scatter.  With
// FX (FP32 only) the slice holds the integer sums of the fixed-point scatter,
// converted with the scale inv when round 0 reads them.
template <typename T, int L, int LE, int K, bool FX = false>
__device__ __forceinline__ void fwht_rounds(T *Sg, T (&v)[1 << LE], int q, int g,
                                            float inv = 1.f) {
    using S = FwhtShape<T, L, LE>;
    using RK = typename S::template Round<K>;
    constexpr int E = S::E;
    // FP32 transforms of more than one round zero the slice while the last
    // round reads it; the others store zeros after the last round
    constexpr bool kExch = sizeof(T) == 4 && K > 0 && K + 1 == S::NR;
    T *base = Sg + RK::addr(q, 0);
    if constexpr (FX && K == 0) {
        static_assert(sizeof(T) == 4, "fixed-point scatter is FP32 only");
        round_load_fixed<L, LE>(base, v, inv);
    } else if constexpr (kExch) {
        round_load_clear<T, L, LE, K>(base, v);
    } else {
        round_load<T, L, LE, K>(base, v);
    }
    reg_fwht_any<T, E, RK::nb>(v);
    if constexpr (K + 1 < S::NR) {
        round_store<T, L, LE, K>(base, v);
        group_sync<S::P>(g);
        fwht_rounds<T, L, LE, K + 1>(Sg, v, q, g);
    } else if constexpr (!kExch) {
        T zero[E];
#pragma unroll
        for (int j = 0; j < E; ++j) zero[j] = T(0);
        round_store<T, L, LE, K>(base, zero);
    }
}

// index (in the unpadded slice) of register j of thread q after the last round
template <typename T, int L, int LE>
__device__ __forceinline__ int final_index(int q, int j) {
    using S = FwhtShape<T, L, LE>;
    return S::template Round<S::NR - 1>::u(q, j);
}

// top bits of (a x + c) mod 2^64: the multiply-add-shift hash of Sec. 4.2
__device__ __forceinline__ uint32_t mas_hash(uint64_t a, uint64_t c, uint64_t x, int shift) {
    return (uint32_t)((a * x + c) >> shift);
}

__device__ __forceinline__ uint32_t mas_sign_bit(uint64_t a, uint64_t c, uint64_t x) {
    return (uint32_t)((a * x + c) >> 63);   // 1 means the sign -1
}

// (a x + c) mod 2^64 along x0, x0 + D, x0 + 2 D, ...: one 64-bit add per step
// instead of a multiply (the same values as mas_hash and mas_sign_bit)
struct MasWalk {
    uint64_t v, step;
    __device__ __forceinline__ MasWalk(uint64_t a, uint64_t c, uint64_t x0, uint64_t d)
        : v(a * x0 + c), step(a * d) {}
    __device__ __forceinline__ uint32_t top(int shift) const { return (uint32_t)(v >> shift); }
    __device__ __forceinline__ void next() { v += step; }
};

}  // namespace cmm
