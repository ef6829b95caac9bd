// adjoint.cu -- backward pass of the mean-over-d estimator at a list of pairs.
//
// Forward (not in the paper's code; the unbiased single-repetition estimate of
// Sec. 3.1 averaged over r):  Chat[i][j] = (1/d) sum_r s1_r(i) s2_r(j) R_r[h1_r(i) XOR h2_r(j)],
// with R_r = sum_t x_{r,t} XOR-conv y_{r,t} (Algorithm 1, Sec. 3.2).  For a loss
// sum_q W_q Chat[I_q][J_q] the estimator is bilinear in (A, B), and with
//     G_r[w] = (1/d) sum_{q : h1_r(I_q) XOR h2_r(J_q) = w} W_q s1_r(I_q) s2_r(J_q)
// the gradients are
//     dA[i][t] = s1_r(i) sum_r (G_r XOR-conv y_{r,t})[h1_r(i)],
//     dB[t][j] = s2_r(j) sum_r (G_r XOR-conv x_{r,t})[h2_r(j)],
// and each XOR convolution is (1/b) H((H G_r) o (H y_{r,t})) (Sec. 3.2).
//
// With FP32 butterflies the two scatters are the fixed-point scatter of the
// sketch kernel (integer bucket sums, per-column power-of-two scales from the
// column maxima, bucket occupancy counted once per CTA and repetition).
//
// Kernels: adj_g_kernel scatters the weights into G (FP64); the FP64 finish
// pass turns G into Gs = (1/b) H G; adjoint_kernel then, per (t, r) and per
// frequency slice, rebuilds H x and H y exactly as the sketch kernel does,
// multiplies each by Gs, transforms back and gathers the result at the rows'
// and columns' buckets into a shared-memory dA column / dB row.
#include "cmm_internal.h"
#include "fwht_device.cuh"
#include "sketch_impl.cuh"

namespace cmm {

namespace {

__global__ void adj_g_kernel(const __grid_constant__ HashParams hp, int d, int L, int64_t P,
                             const int32_t *__restrict__ I, const int32_t *__restrict__ J,
                             const double *__restrict__ W, double *__restrict__ G) {
    const int64_t b = (int64_t)1 << L;
    const int shift = 64 - L;
    const int64_t n = P * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / P);
        const int64_t q = e % P;
        const HashRep &h = hp.rep[r];
        const uint64_t i = (uint64_t)I[q], j = (uint64_t)J[q];
        const uint32_t w = (uint32_t)((h.a1 * i + h.c1) >> shift) ^ (uint32_t)((h.a2 * j + h.c2) >> shift);
        const uint64_t neg = ((h.as1 * i + h.cs1) >> 63) ^ ((h.as2 * j + h.cs2) >> 63);
        const double v = (neg ? -W[q] : W[q]) / d;
        atomicAdd(G + r * b + w, v);
    }
}

// gather the transformed slice at the buckets of one column of keys and add
// into acc[x] (thread q owns x = q, q + P, ...)
template <typename T, int L, int LE>
__device__ __forceinline__ void gather_keys(const T *Sg, T *acc, int64_t n, uint64_t a, uint64_t c,
                                            uint64_t as, uint64_t cs, int shift, uint32_t u_hi,
                                            int q) {
    using S = FwhtShape<T, L, LE>;
    MasWalk hw(a, c, (uint64_t)q, S::P), sw(as, cs, (uint64_t)q, S::P);
    for (int64_t x = q; x < n; x += S::P, hw.next(), sw.next()) {
        const uint32_t h = hw.top(shift);
        const uint32_t neg = sw.top(63) ^ (__popc((h >> L) & u_hi) & 1u);
        const T v = Sg[pad_index<T, L, LE>((int)(h & (S::N - 1)))];
        acc[x] += neg ? -v : v;
    }
}

template <typename T, int L, int LE, int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
adjoint_kernel(const T *__restrict__ At, int64_t ldat, const T *__restrict__ Bp, int64_t ldbp,
               int64_t m, int64_t k, int64_t p, int Lfull, int C, int64_t chunk, int d,
               const __grid_constant__ HashParams hp, const double *__restrict__ Gs,
               const float *__restrict__ colmax, T *__restrict__ dAt, T *__restrict__ dBt,
               int accumulate) {
    using S = FwhtShape<T, L, LE>;
    constexpr int E = S::E, P = S::P, G = THREADS / P;
    constexpr bool FX = sizeof(T) == 4;   // fixed-point scatter
    __shared__ int s_red[32];
    __shared__ int s_cmax[2 * CMM_MAX_D];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int tid = threadIdx.x;
    const int g = tid / P, q = tid % P;
    T *Sg = sm + g * S::STRIDE;
    T *dAc = sm + G * S::STRIDE + g * m;
    T *dBr = sm + G * S::STRIDE + G * m + g * p;

    const uint32_t u_hi = (uint32_t)(blockIdx.x % C);
    const int64_t blk = blockIdx.x / C;
    const int64_t t0 = blk * chunk;
    const int64_t t1 = (t0 + chunk < k) ? t0 + chunk : k;
    const int shift = 64 - Lfull;
    const int64_t b = (int64_t)1 << Lfull;

    for (int i = tid; i < G * S::STRIDE; i += THREADS) sm[i] = T(0);
    __syncthreads();
    if constexpr (FX) {
        int *S0 = reinterpret_cast<int *>(sm);
        for (int r = 0; r < d; ++r) {
            const HashRep &H = hp.rep[r];
            const int ca = block_cmax<L, LE, THREADS>(S0, nullptr, m, H.a1, H.c1, shift, s_red);
            const int cb = block_cmax<L, LE, THREADS>(S0, nullptr, p, H.a2, H.c2, shift, s_red);
            if (tid == 0) {
                s_cmax[r] = ca;
                s_cmax[CMM_MAX_D + r] = cb;
            }
        }
        __syncthreads();
    }
    int *Sgi = reinterpret_cast<int *>(Sg);

    T xh[E], v[E], gh[E];
    const int64_t nt = t1 > t0 ? t1 - t0 : 0;
    const int64_t iters = (nt + G - 1) / G;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t t = t0 + it * G + g;
        const bool active = t < t1;
        for (int64_t x = q; x < m; x += P) dAc[x] = T(0);
        for (int64_t x = q; x < p; x += P) dBr[x] = T(0);
        for (int r = 0; r < d; ++r) {
            const HashRep H = hp.rep[r];
            // H x_t and H y_t of this slice, as in the sketch kernel
            float sA = 1.f, invA = 1.f, sB = 1.f, invB = 1.f;
            if constexpr (FX) {
                if (active) {
                    fixed_scale(__ldg(colmax + t), s_cmax[r], sA, invA);
                    fixed_scale(__ldg(colmax + k + t), s_cmax[CMM_MAX_D + r], sB, invB);
                    scatter_column_fixed<L, LE>(Sgi, (const float *)(At + t * ldat), m, H.a1,
                                                H.c1, H.as1, H.cs1, shift, u_hi, q, sA);
                }
            } else if (active) {
                scatter_column<T, L, LE>(Sg, At + t * ldat, m, H.a1, H.c1, H.as1, H.cs1, shift,
                                         u_hi, q);
            }
            group_sync<P>(g);
            fwht_rounds<T, L, LE, 0, FX>(Sg, v, q, g, invA);
#pragma unroll
            for (int j = 0; j < E; ++j) xh[j] = v[j];
            group_sync<P>(g);
            if constexpr (FX) {
                if (active)
                    scatter_column_fixed<L, LE>(Sgi, (const float *)(Bp + t * ldbp), p, H.a2,
                                                H.c2, H.as2, H.cs2, shift, u_hi, q, sB);
            } else if (active) {
                scatter_column<T, L, LE>(Sg, Bp + t * ldbp, p, H.a2, H.c2, H.as2, H.cs2, shift,
                                         u_hi, q);
            }
            group_sync<P>(g);
            fwht_rounds<T, L, LE, 0, FX>(Sg, v, q, g, invB);
            const double *gr = Gs + r * b + (int64_t)u_hi * S::N;
#pragma unroll
            for (int j = 0; j < E; ++j) gh[j] = (T)__ldg(gr + final_index<T, L, LE>(q, j));
            // dA: H((1/b) H G o H y), gathered at h1(i)
#pragma unroll
            for (int j = 0; j < E; ++j) Sg[pad_index<T, L, LE>(final_index<T, L, LE>(q, j))] = gh[j] * v[j];
            group_sync<P>(g);
            fwht_rounds<T, L, LE, 0>(Sg, v, q, g);
#pragma unroll
            for (int j = 0; j < E; ++j) Sg[pad_index<T, L, LE>(final_index<T, L, LE>(q, j))] = v[j];
            group_sync<P>(g);
            if (active) gather_keys<T, L, LE>(Sg, dAc, m, H.a1, H.c1, H.as1, H.cs1, shift, u_hi, q);
            group_sync<P>(g);
            // dB: H((1/b) H G o H x), gathered at h2(j)
#pragma unroll
            for (int j = 0; j < E; ++j) Sg[pad_index<T, L, LE>(final_index<T, L, LE>(q, j))] = gh[j] * xh[j];
            group_sync<P>(g);
            fwht_rounds<T, L, LE, 0>(Sg, v, q, g);
#pragma unroll
            for (int j = 0; j < E; ++j) Sg[pad_index<T, L, LE>(final_index<T, L, LE>(q, j))] = v[j];
            group_sync<P>(g);
            if (active) gather_keys<T, L, LE>(Sg, dBr, p, H.a2, H.c2, H.as2, H.cs2, shift, u_hi, q);
            group_sync<P>(g);
#pragma unroll
            for (int j = 0; j < E; ++j) Sg[pad_index<T, L, LE>(final_index<T, L, LE>(q, j))] = T(0);
            group_sync<P>(g);
        }
        if (active) {
            T *da = dAt + t * m;
            T *db = dBt + t * p;
            if (accumulate) {
                for (int64_t x = q; x < m; x += P) atomicAdd(da + x, dAc[x]);
                for (int64_t x = q; x < p; x += P) atomicAdd(db + x, dBr[x]);
            } else {
                for (int64_t x = q; x < m; x += P) da[x] = dAc[x];
                for (int64_t x = q; x < p; x += P) db[x] = dBr[x];
            }
        }
    }
}

template <typename T, int L, int LE, int THREADS>
cudaError_t launch_adj_inst(const AdjointPlan &pl, const T *At, const T *Bp, int64_t m, int64_t k,
                            int64_t p, int d, const HashParams &hp, const double *Gs,
                            const float *colmax, T *dAt, T *dBt, cudaStream_t s) {
    auto kern = adjoint_kernel<T, L, LE, THREADS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pl.smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)((int64_t)pl.nchunks * pl.C), THREADS, pl.smem, s>>>(
        At, pl.ldat, Bp, pl.ldbp, m, k, p, pl.L, pl.C, pl.chunk, d, hp, Gs, colmax, dAt, dBt,
        pl.C > 1 ? 1 : 0);
    return cudaGetLastError();
}

template <typename T> struct AdjCfg;
template <> struct AdjCfg<float> { static constexpr int LEmax = 5, Lmax = kMaxLloF32; };
template <> struct AdjCfg<double> { static constexpr int LEmax = 4, Lmax = kMaxLloF64; };

template <typename T, int L>
constexpr int adj_threads() {
    constexpr int LE = L < AdjCfg<T>::LEmax ? L : AdjCfg<T>::LEmax;
    constexpr int P = (1 << L) >> LE;
    return P >= 256 ? P : 256;
}

template <typename T, int L>
cudaError_t run_adj(const AdjointPlan &pl, const T *At, const T *Bp, int64_t m, int64_t k, int64_t p,
                    int d, const HashParams &hp, const double *Gs, const float *colmax, T *dAt,
                    T *dBt, cudaStream_t s) {
    constexpr int LE = L < AdjCfg<T>::LEmax ? L : AdjCfg<T>::LEmax;
    return launch_adj_inst<T, L, LE, adj_threads<T, L>()>(pl, At, Bp, m, k, p, d, hp, Gs, colmax,
                                                          dAt, dBt, s);
}

}  // namespace

int adjoint_threads(int prec, int Llo) {
    if (prec == CMM_PREC_F64) {
        switch (Llo) {
#define CASE(L) case L: return adj_threads<double, L>();
            CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10)
            CASE(11) CASE(12) CASE(13)
#undef CASE
        }
        return 0;
    }
    switch (Llo) {
#define CASE(L) case L: return adj_threads<float, L>();
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10)
        CASE(11) CASE(12) CASE(13) CASE(14)
#undef CASE
    }
    return 0;
}

cudaError_t launch_adj_g(const HashParams &hp, int d, int L, int64_t P, const int32_t *I,
                         const int32_t *J, const double *W, double *G, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(G, 0, (size_t)d * ((size_t)1 << L) * sizeof(double), s);
    if (e != cudaSuccess || P == 0) return e;
    int64_t blocks = (P * d + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    adj_g_kernel<<<(unsigned)blocks, 256, 0, s>>>(hp, d, L, P, I, J, W, G);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const AdjointPlan &pl, const void *At, const void *Bp, int64_t m,
                           int64_t k, int64_t p, int d, const HashParams &hp, const double *Gs,
                           const float *colmax, void *dAt, void *dBt, cudaStream_t s) {
    if (pl.C > 1) {
        const size_t es = pl.prec == CMM_PREC_F64 ? 8 : 4;
        cudaError_t e = cudaMemsetAsync(dAt, 0, (size_t)k * m * es, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(dBt, 0, (size_t)k * p * es, s);
        if (e != cudaSuccess) return e;
    }
    if (pl.prec == CMM_PREC_F64) {
        const double *a = (const double *)At, *bb = (const double *)Bp;
        double *da = (double *)dAt, *db = (double *)dBt;
        switch (pl.Llo) {
#define CASE(L) case L: return run_adj<double, L>(pl, a, bb, m, k, p, d, hp, Gs, nullptr, da, db, s);
            CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10)
            CASE(11) CASE(12) CASE(13)
#undef CASE
        }
        return cudaErrorInvalidValue;
    }
    const float *a = (const float *)At, *bb = (const float *)Bp;
    float *da = (float *)dAt, *db = (float *)dBt;
    switch (pl.Llo) {
#define CASE(L) case L: return run_adj<float, L>(pl, a, bb, m, k, p, d, hp, Gs, colmax, da, db, s);
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10)
        CASE(11) CASE(12) CASE(13) CASE(14)
#undef CASE
    }
    return cudaErrorInvalidValue;
}

}  // namespace cmm
