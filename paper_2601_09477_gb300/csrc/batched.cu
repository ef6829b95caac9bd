// batched.cu -- many independent problems in one persistent launch.
//
// Every problem q (A_q m_q x k_q, B_q k_q x p_q, sketch length b_q = 2^L_q,
// its own hash functions, the shared d) runs the whole path of Algorithm 1:
// Compress (sketch tasks: one per repetition r, frequency slice u_hi and block
// of inner indices, exactly the CTA body of the single-problem sketch kernel),
// the FP64 finish (one task per (q, r): reduction over blocks, inverse
// transform, 1/b), and Decompress of every entry (one task per tile of rows).
//
// The sketch scatters in fixed point (one power-of-two scale per column, see
// sketch_impl.cuh), which needs the maxima |A^T[t][:]| and |B[t][:]| of every
// column first: column-maximum tasks (rows of A^T and B in blocks) come first
// in the task list.
//
// The task list is ordered column-maximum tasks, sketch tasks of all problems,
// then finish tasks, then extraction tasks.  CTAs (one per SM) take tasks from
// an atomic counter.  A sketch task waits until the column maxima of its
// problem are done, a finish task until all sketch tasks of its (q, r) are
// done and an extraction task until all d finish tasks of q are done; the waits
// are bounded (a globaltimer budget): on expiry the kernel sets an error word,
// every CTA stops taking tasks, and cmm_batched_status returns
// CMM_ERR_TIMEOUT.  Because every task is dequeued after all tasks it depends
// on and sketch tasks wait on nothing, the waits always end in a correct run.
//
// The per-CTA slice (b-tile, 2^Llo) and the block of inner indices per task
// (t-tile) come from the caller (the autotuner) or a default rule.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "cmm_internal.h"
#include "extract_device.cuh"
#include "fwht_device.cuh"
#include "sketch_impl.cuh"

namespace cmm {

namespace {

constexpr int kBThreads = 512;
constexpr int kBMinLlo = 5;
constexpr int kBMaxLlo = 14;
constexpr int kBFinishLf = 12;
constexpr size_t kBSmem = 160 * 1024;
constexpr int kExTileRows = 32;
constexpr int kCmRows = 64;   // rows of A^T / B per column-maximum task
constexpr unsigned long long kDefaultWaitNs = 4000000000ULL;   // 4 s

struct BProblem {
    const float *At;
    int64_t ldat;
    const float *Bp;
    int64_t ldbp;
    int64_t m, k, p;
    int L, Llo, C, nchunks;
    int64_t chunk;
    double *partial, *Z, *R, *Cout;
    int64_t ldc;
    float *cm;      // column maxima: A^T rows [0, k), then B rows [k, 2k)
    int hash_off;
    int ex_tiles;
    int cm_tasks;
};

struct BTask {
    int32_t type;   // 0 sketch, 1 finish, 2 extract, 3 column maxima
    int32_t prob;
    int32_t a;      // sketch: r * C + u_hi; finish: r; extract: row tile; maxima: row block
    int32_t b;      // sketch: block of inner indices
};

// counters: [0] next task, [1] error word, then done_sketch[Q * d],
// done_finish[Q], done_cm[Q]
struct BCounters {
    int *next, *err, *done_sketch, *done_finish, *done_cm;
};

__device__ __forceinline__ int load_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// thread 0 waits (bounded) until *ctr >= target; returns false on timeout or
// when another CTA has already raised the error word
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ bool wait_for(const int *ctr, int target, int *err, int *s_flag,
                         unsigned long long budget_ns) {
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long t0 = global_ns();
        while (load_acquire(ctr) < target) {
            if (load_acquire(err) != 0) { ok = 0; break; }
            if (global_ns() - t0 > budget_ns) {
                atomicExch(err, 1);
                ok = 0;
                break;
            }
            __nanosleep(200);
        }
        __threadfence();
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

__device__ __forceinline__ void signal_done(int *ctr) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1);
    }
}

template <int L>
__device__ __forceinline__ void sketch_task(const BProblem &pr, const HashRep &H, int a, int blk,
                                            int d, unsigned char *smem) {
    constexpr int LE = L < 5 ? L : 5;
    const uint32_t u_hi = (uint32_t)(a % pr.C);
    const int r = a / pr.C;
    const int64_t t0 = (int64_t)blk * pr.chunk;
    const int64_t t1 = (t0 + pr.chunk < pr.k) ? t0 + pr.chunk : pr.k;
    const int64_t b = (int64_t)1 << pr.L;
    double *out = pr.partial + ((int64_t)blk * d + r) * b + (int64_t)u_hi * (1 << L);
    sketch_block<float, float, L, LE, kBThreads, true>(pr.At, pr.ldat, pr.Bp, pr.ldbp, pr.m, pr.p,
                                                       pr.L, u_hi, t0, t1, H, nullptr, nullptr,
                                                       pr.cm, pr.cm + pr.k, out, smem);
}

// max |x| over rows [blk * kCmRows, ...) of A^T (rows < k) and B (rows >= k)
__device__ void colmax_task(const BProblem &pr, int blk) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = (int64_t)blk * kCmRows;
    const int64_t r1 = r0 + kCmRows < 2 * pr.k ? r0 + kCmRows : 2 * pr.k;
    for (int64_t r = r0 + warp; r < r1; r += kBThreads / 32) {
        const bool isA = r < pr.k;
        const float *row = isA ? pr.At + r * pr.ldat : pr.Bp + (r - pr.k) * pr.ldbp;
        const int64_t n = isA ? pr.m : pr.p;
        float mx = 0.f;
        for (int64_t c = lane; c < n; c += 32) mx = fmaxf(mx, fabsf(__ldcs(row + c)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) pr.cm[r] = mx;
    }
}

__device__ void dispatch_sketch(const BProblem &pr, const HashRep &H, int a, int blk, int d,
                                unsigned char *smem) {
    switch (pr.Llo) {
        case 5: sketch_task<5>(pr, H, a, blk, d, smem); break;
        case 6: sketch_task<6>(pr, H, a, blk, d, smem); break;
        case 7: sketch_task<7>(pr, H, a, blk, d, smem); break;
        case 8: sketch_task<8>(pr, H, a, blk, d, smem); break;
        case 9: sketch_task<9>(pr, H, a, blk, d, smem); break;
        case 10: sketch_task<10>(pr, H, a, blk, d, smem); break;
        case 11: sketch_task<11>(pr, H, a, blk, d, smem); break;
        case 12: sketch_task<12>(pr, H, a, blk, d, smem); break;
        case 13: sketch_task<13>(pr, H, a, blk, d, smem); break;
        case 14: sketch_task<14>(pr, H, a, blk, d, smem); break;
        default: break;
    }
}

// in-place FWHT of n doubles at stride `st` (n * st <= smem), all threads
__device__ void smem_fwht(double *v, int n, int st, int cols) {
    for (int h = 1; h < n; h <<= 1) {
        for (int e = threadIdx.x; e < (n / 2) * cols; e += kBThreads) {
            const int pair = e / cols, c = e % cols;
            const int lo = (pair / h) * 2 * h + (pair % h);
            const double x = v[lo * st + c], y = v[(lo + h) * st + c];
            v[lo * st + c] = x + y;
            v[(lo + h) * st + c] = x - y;
        }
        __syncthreads();
    }
}

// (q, r): R_r = (1/b) H sum_blocks partial, FP64
__device__ void finish_task(const BProblem &pr, int r, int d, double *sm) {
    const int L = pr.L;
    const int64_t b = (int64_t)1 << L;
    const int Lf = L < kBFinishLf ? L : kBFinishLf;
    const int Nf = 1 << Lf;
    const int Ch = (int)(b >> Lf);
    const int64_t stride = (int64_t)d * b;
    const double *src = pr.partial + (int64_t)r * b;
    const double inv_b = ldexp(1.0, -L);
    for (int rr = 0; rr < Ch; ++rr) {
        for (int e = threadIdx.x; e < Nf; e += kBThreads) {
            double s = 0.0;
            for (int c = 0; c < pr.nchunks; ++c) s += src[(int64_t)c * stride + (int64_t)rr * Nf + e];
            sm[e] = s;
        }
        __syncthreads();
        smem_fwht(sm, Nf, 1, 1);
        for (int e = threadIdx.x; e < Nf; e += kBThreads) {
            if (Ch == 1)
                pr.R[(int64_t)r * b + e] = sm[e] * inv_b;
            else
                pr.Z[(int64_t)r * b + (int64_t)rr * Nf + e] = sm[e];
        }
        __syncthreads();
    }
    if (Ch > 1) {
        __threadfence_block();
        const int W = (4096 / Ch) < 1 ? 1 : ((4096 / Ch) > Nf ? Nf : 4096 / Ch);
        for (int c0 = 0; c0 < Nf; c0 += W) {
            for (int e = threadIdx.x; e < Ch * W; e += kBThreads) {
                const int rr = e / W, c = e % W;
                sm[e] = pr.Z[(int64_t)r * b + (int64_t)rr * Nf + c0 + c];
            }
            __syncthreads();
            smem_fwht(sm, Ch, W, W);
            for (int e = threadIdx.x; e < Ch * W; e += kBThreads) {
                const int rr = e / W, c = e % W;
                pr.R[(int64_t)r * b + (int64_t)rr * Nf + c0 + c] = sm[e] * inv_b;
            }
            __syncthreads();
        }
    }
}

// value of one repetition, from R in shared (staged) or global memory
__device__ __forceinline__ long long rep_key_any(const double *Rr, uint32_t h1, uint32_t h2,
                                                 uint32_t mask) {
    const uint32_t x = h1 ^ h2;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(Rr[x & mask]) ^
                                    ((unsigned long long)(x >> 31) << 63);
    return key_of_bits(bits);
}

// Decompress rows [tile * kExTileRows, ...) of problem q (median over d, D = d
// at compile time or 0 for the generic path)
template <int D>
__device__ void extract_task(const BProblem &pr, const HashRep *hashes, int tile, int d,
                             unsigned char *smem) {
    const int64_t b = (int64_t)1 << pr.L;
    const uint32_t mask = (uint32_t)(b - 1);
    const int shift = 64 - pr.L;
    const size_t rbytes = (size_t)d * b * sizeof(double);
    uint32_t *h1s = reinterpret_cast<uint32_t *>(smem);                 // [kExTileRows][d]
    double *Rs = reinterpret_cast<double *>(smem + 16384);
    const bool staged = rbytes + 16384 <= kBSmem;
    const double *Rsrc = staged ? Rs : pr.R;
    if (staged)
        for (int64_t e = threadIdx.x; e < (int64_t)d * b; e += kBThreads) Rs[e] = pr.R[e];
    const int64_t i0 = (int64_t)tile * kExTileRows;
    for (int e = threadIdx.x; e < kExTileRows * d; e += kBThreads) {
        const int rr = e / d, r = e % d;
        const uint64_t i = (uint64_t)(i0 + rr);
        const HashRep &H = hashes[pr.hash_off + r];
        const uint32_t bk = (uint32_t)((H.a1 * i + H.c1) >> shift);
        const uint32_t sg = (uint32_t)((H.as1 * i + H.cs1) >> 63);
        h1s[rr * d + r] = bk | (sg << 31);
    }
    __syncthreads();
    for (int64_t j = threadIdx.x; j < pr.p; j += kBThreads) {
        uint32_t h2v[D > 0 ? D : CMM_MAX_D];
        const int dd = D > 0 ? D : d;
#pragma unroll
        for (int r = 0; r < dd; ++r) {
            const HashRep &H = hashes[pr.hash_off + r];
            const uint32_t bk = (uint32_t)((H.a2 * (uint64_t)j + H.c2) >> shift);
            const uint32_t sg = (uint32_t)((H.as2 * (uint64_t)j + H.cs2) >> 63);
            h2v[r] = bk | (sg << 31);
        }
        for (int rr = 0; rr < kExTileRows && i0 + rr < pr.m; ++rr) {
            double est;
            if constexpr (D > 0) {
                long long v[D];
#pragma unroll
                for (int r = 0; r < D; ++r) v[r] = rep_key_any(Rsrc + r * b, h1s[rr * d + r], h2v[r], mask);
                est = val_of_key(median_odd<D>(v));
            } else {
                long long v[CMM_MAX_D];
                for (int r = 0; r < d; ++r) v[r] = rep_key_any(Rsrc + r * b, h1s[rr * d + r], h2v[r], mask);
                est = combine_generic(v, d, CMM_MEDIAN);
            }
            pr.Cout[(i0 + rr) * pr.ldc + j] = est;
        }
    }
}

template <int D>
__global__ void __launch_bounds__(kBThreads, 1)
batched_kernel(const BTask *__restrict__ tasks, int ntasks, const BProblem *__restrict__ probs,
               const HashRep *__restrict__ hashes, int d, BCounters ctr,
               unsigned long long budget_ns, int extra_target) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_task, s_flag;
    for (;;) {
        if (threadIdx.x == 0) s_task = load_acquire(ctr.err) ? ntasks : atomicAdd(ctr.next, 1);
        __syncthreads();
        const int tid = s_task;
        __syncthreads();
        if (tid >= ntasks) break;
        const BTask tk = tasks[tid];
        const BProblem &pr = probs[tk.prob];
        if (tk.type == 3) {
            colmax_task(pr, tk.a);
            signal_done(ctr.done_cm + tk.prob);
        } else if (tk.type == 0) {
            if (!wait_for(ctr.done_cm + tk.prob, pr.cm_tasks, ctr.err, &s_flag, budget_ns)) break;
            const int r = tk.a / pr.C;
            dispatch_sketch(pr, hashes[pr.hash_off + r], tk.a, tk.b, d, smem_raw);
            signal_done(ctr.done_sketch + tk.prob * d + r);
        } else if (tk.type == 1) {
            if (!wait_for(ctr.done_sketch + tk.prob * d + tk.a, pr.C * pr.nchunks + extra_target,
                          ctr.err, &s_flag, budget_ns))
                break;
            finish_task(pr, tk.a, d, reinterpret_cast<double *>(smem_raw));
            signal_done(ctr.done_finish + tk.prob);
        } else {
            if (!wait_for(ctr.done_finish + tk.prob, d, ctr.err, &s_flag, budget_ns)) break;
            if (pr.Cout) extract_task<D>(pr, hashes, tk.a, d, smem_raw);
            __syncthreads();
        }
    }
}

// host-side plan kept inside the caller's cmm_batch_plan
struct BPlan {
    void *ws;
    size_t ws_bytes;
    int Q, d, ntasks, grid;
    size_t off_ctr, ctr_bytes, off_tasks, off_probs, off_hash;
    unsigned magic;
};
static_assert(sizeof(BPlan) <= sizeof(cmm_batch_plan), "plan does not fit the opaque handle");
constexpr unsigned kPlanMagic = 0xC3B47A11u;

constexpr size_t kAlign = 256;
size_t aup(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// t-tile rule: about 6e7 butterfly-equivalents per sketch task, a multiple of
// the group count, at most k
int64_t default_chunk(int Llo, int64_t k) {
    const int LE = Llo < 5 ? Llo : 5;
    const int P = (1 << Llo) >> LE;
    const int G = kBThreads / P;
    double per_t = (double)(1 << Llo) * (Llo > 0 ? Llo : 1);
    int64_t c = (int64_t)(6.0e7 / per_t);
    c = (c + G - 1) / G * G;
    if (c < G) c = G;
    if (c > k) c = k;
    return c < 1 ? 1 : c;
}

struct Sizes {
    std::vector<int> Llo, C, nchunks;
    std::vector<int64_t> chunk;
    std::vector<size_t> off_part, off_Z, off_At, off_Bp, off_cm;
    size_t total;
    size_t off_ctr, ctr_bytes, off_tasks, off_probs, off_hash;
    int ntasks;
};

int plan_sizes(const cmm_problem *pb, int Q, int d, Sizes &sz) {
    sz.Llo.resize(Q);
    sz.C.resize(Q);
    sz.nchunks.resize(Q);
    sz.chunk.resize(Q);
    sz.off_part.resize(Q);
    sz.off_Z.resize(Q);
    sz.off_At.resize(Q);
    sz.off_Bp.resize(Q);
    sz.off_cm.resize(Q);
    size_t off = 0;
    sz.off_ctr = off;
    sz.ctr_bytes = (size_t)(2 + Q * d + 2 * Q) * sizeof(int);
    off += aup(sz.ctr_bytes);
    int64_t ntasks = 0;
    for (int q = 0; q < Q; ++q) {
        const cmm_problem &P = pb[q];
        int Llo = P.tile_log2 > 0 ? P.tile_log2 : std::min(P.log2b, kBMaxLlo);
        Llo = std::min(Llo, P.log2b);
        if (Llo < kBMinLlo || Llo > kBMaxLlo) return -1;
        sz.Llo[q] = Llo;
        sz.C[q] = 1 << (P.log2b - Llo);
        const int64_t kk = std::max<int64_t>(P.k, 1);
        int64_t ch = P.t_tile > 0 ? std::min<int64_t>(P.t_tile, kk) : default_chunk(Llo, kk);
        sz.chunk[q] = ch;
        sz.nchunks[q] = (int)((kk + ch - 1) / ch);
        const int64_t tiles = (P.m + kExTileRows - 1) / kExTileRows;
        ntasks += (int64_t)d * sz.C[q] * sz.nchunks[q] + d + (P.C ? tiles : 0) +
                  (2 * P.k + kCmRows - 1) / kCmRows;
    }
    if (ntasks > 0x7fffffff) return -2;
    sz.ntasks = (int)ntasks;
    sz.off_tasks = off;
    off += aup((size_t)ntasks * sizeof(BTask));
    sz.off_probs = off;
    off += aup((size_t)Q * sizeof(BProblem));
    sz.off_hash = off;
    off += aup((size_t)Q * d * sizeof(HashRep));
    for (int q = 0; q < Q; ++q) {
        const cmm_problem &P = pb[q];
        const size_t b = (size_t)1 << P.log2b;
        sz.off_At[q] = off;
        sz.off_Bp[q] = off;   // A^T and B are read in place (FP32, row-major)
        sz.off_part[q] = off;
        off += aup((size_t)sz.nchunks[q] * d * b * sizeof(double));
        sz.off_Z[q] = off;
        off += aup((size_t)d * b * sizeof(double));
        sz.off_cm[q] = off;
        off += aup((size_t)2 * P.k * sizeof(float));
    }
    sz.total = off;
    return 0;
}

int check_problems(const cmm_problem *pb, int Q, int d, int dtype, int prec) {
    char msg[256];
    if (!pb || Q < 1) return set_error(CMM_ERR_ARG, "batched: no problems");
    if (d < 1 || d > CMM_MAX_D) return set_error(CMM_ERR_RANGE, "batched: d outside [1, 64]");
    if (dtype != CMM_F32 || prec != CMM_PREC_F32)
        return set_error(CMM_ERR_ARG, "batched: FP32 operands and FP32 butterflies only");
    for (int q = 0; q < Q; ++q) {
        const cmm_problem &P = pb[q];
        if (P.m < 1 || P.k < 0 || P.p < 1 || P.m >= (1LL << 31) || P.p >= (1LL << 31) ||
            P.log2b < kBMinLlo || P.log2b > CMM_MAX_LOG2B || !P.hash_params || !P.R ||
            (P.k > 0 && (!P.A || !P.B)) || P.transA != 1 ||
            P.lda < (P.transA ? P.m : P.k) || P.ldb < P.p || (P.C && P.ldc < P.p) ||
            P.tile_log2 < 0 || P.tile_log2 > kBMaxLlo || P.t_tile < 0) {
            std::snprintf(msg, sizeof msg, "batched: problem %d has invalid sizes or pointers", q);
            return set_error(P.log2b > CMM_MAX_LOG2B || P.log2b < kBMinLlo ? CMM_ERR_RANGE : CMM_ERR_ARG,
                             msg);
        }
    }
    return CMM_OK;
}

}  // namespace

}  // namespace cmm

using namespace cmm;

extern "C" size_t cmm_batched_workspace_bytes(const cmm_problem *problems, int32_t Q, int32_t d,
                                              int32_t dtype, int32_t prec) {
    if (check_problems(problems, Q, d, dtype, prec) != CMM_OK) return 0;
    Sizes sz;
    if (plan_sizes(problems, Q, d, sz) != 0) return 0;
    return sz.total;
}

extern "C" int cmm_batched_prepare(const cmm_problem *problems, int32_t Q, int32_t d,
                                   int32_t dtype, int32_t prec, void *ws, size_t ws_bytes,
                                   cmm_batch_plan *plan, void *stream) {
    int rc = check_problems(problems, Q, d, dtype, prec);
    if (rc) return rc;
    if (!plan) return set_error(CMM_ERR_ARG, "batched: plan is NULL");
    Sizes sz;
    if (plan_sizes(problems, Q, d, sz) != 0)
        return set_error(CMM_ERR_RANGE, "batched: tile sizes out of range or too many tasks");
    if (!ws || reinterpret_cast<uintptr_t>(ws) % kAlign || ws_bytes < sz.total) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "batched: workspace needs %zu bytes, 256-byte aligned", sz.total);
        return set_error(CMM_ERR_WORKSPACE, msg);
    }
    char *base = static_cast<char *>(ws);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<BProblem> probs(Q);
    std::vector<HashRep> hashes((size_t)Q * d);
    std::vector<BTask> tasks;
    tasks.reserve(sz.ntasks);
    for (int q = 0; q < Q; ++q) {
        const cmm_problem &P = problems[q];
        BProblem &bp = probs[q];
        bp.At = (const float *)P.A;
        bp.ldat = P.lda;
        bp.Bp = (const float *)P.B;
        bp.ldbp = P.ldb;
        bp.m = P.m;
        bp.k = P.k;
        bp.p = P.p;
        bp.L = P.log2b;
        bp.Llo = sz.Llo[q];
        bp.C = sz.C[q];
        bp.nchunks = sz.nchunks[q];
        bp.chunk = sz.chunk[q];
        bp.partial = reinterpret_cast<double *>(base + sz.off_part[q]);
        bp.Z = reinterpret_cast<double *>(base + sz.off_Z[q]);
        bp.R = P.R;
        bp.Cout = P.C;
        bp.ldc = P.ldc;
        bp.cm = reinterpret_cast<float *>(base + sz.off_cm[q]);
        bp.hash_off = q * d;
        bp.ex_tiles = (int)((P.m + kExTileRows - 1) / kExTileRows);
        bp.cm_tasks = (int)((2 * P.k + kCmRows - 1) / kCmRows);
        for (int r = 0; r < d; ++r) {
            const uint64_t *w = P.hash_params + 8 * r;
            hashes[(size_t)q * d + r] = HashRep{w[0], w[1], w[2], w[3], w[4], w[5], w[6], w[7]};
        }
    }
    // sketch tasks, largest problems first within the phase, then finish, then extract
    std::vector<int> order(Q);
    for (int q = 0; q < Q; ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const double wx = (double)probs[x].k * (1 << probs[x].L) * probs[x].L;
        const double wy = (double)probs[y].k * (1 << probs[y].L) * probs[y].L;
        return wx > wy;
    });
    for (int q : order)
        for (int c = 0; c < probs[q].cm_tasks; ++c) tasks.push_back(BTask{3, q, c, 0});
    for (int q : order)
        for (int c = 0; c < probs[q].nchunks; ++c)
            for (int a = 0; a < d * probs[q].C; ++a) tasks.push_back(BTask{0, q, a, c});
    for (int q : order)
        for (int r = 0; r < d; ++r) tasks.push_back(BTask{1, q, r, 0});
    for (int q : order)
        if (probs[q].Cout)
            for (int t = 0; t < probs[q].ex_tiles; ++t) tasks.push_back(BTask{2, q, t, 0});
    cudaError_t e = cudaMemcpyAsync(base + sz.off_tasks, tasks.data(), tasks.size() * sizeof(BTask),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + sz.off_probs, probs.data(), probs.size() * sizeof(BProblem),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + sz.off_hash, hashes.data(), hashes.size() * sizeof(HashRep),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host vectors go out of scope
    if (e != cudaSuccess) return set_error(CMM_ERR_CUDA, cudaGetErrorString(e));
    BPlan bp{};
    bp.ws = ws;
    bp.ws_bytes = ws_bytes;
    bp.Q = Q;
    bp.d = d;
    bp.ntasks = (int)tasks.size();
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    bp.grid = nsm;
    bp.off_ctr = sz.off_ctr;
    bp.ctr_bytes = sz.ctr_bytes;
    bp.off_tasks = sz.off_tasks;
    bp.off_probs = sz.off_probs;
    bp.off_hash = sz.off_hash;
    bp.magic = kPlanMagic;
    std::memset(plan, 0, sizeof *plan);
    std::memcpy(plan, &bp, sizeof bp);
    return CMM_OK;
}

namespace {
template <int D>
cudaError_t launch_batched_inst(const BPlan &bp, unsigned long long budget_ns, int extra,
                                cudaStream_t s) {
    char *base = static_cast<char *>(bp.ws);
    int *ctr = reinterpret_cast<int *>(base + bp.off_ctr);
    BCounters c{ctr, ctr + 1, ctr + 2, ctr + 2 + bp.Q * bp.d, ctr + 2 + bp.Q * bp.d + bp.Q};
    auto kern = batched_kernel<D>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBSmem);
    if (e != cudaSuccess) return e;
    kern<<<bp.grid, kBThreads, kBSmem, s>>>(reinterpret_cast<const BTask *>(base + bp.off_tasks),
                                            bp.ntasks, reinterpret_cast<const BProblem *>(base + bp.off_probs),
                                            reinterpret_cast<const HashRep *>(base + bp.off_hash), bp.d, c,
                                            budget_ns, extra);
    return cudaGetLastError();
}
}  // namespace

extern "C" int cmm_batched_launch(const cmm_batch_plan *plan, void *stream) {
    return cmm_batched_launch_opts(plan, 0, 0, stream);
}

extern "C" int cmm_batched_launch_opts(const cmm_batch_plan *plan, int64_t wait_budget_us,
                                       int32_t unmet_dependency, void *stream) {
    if (!plan) return set_error(CMM_ERR_ARG, "batched: plan is NULL");
    if (wait_budget_us < 0) return set_error(CMM_ERR_ARG, "batched: negative wait budget");
    const unsigned long long budget_ns =
        wait_budget_us > 0 ? (unsigned long long)wait_budget_us * 1000ULL : kDefaultWaitNs;
    const int extra = unmet_dependency ? 1 : 0;
    BPlan bp;
    std::memcpy(&bp, plan, sizeof bp);
    if (bp.magic != kPlanMagic) return set_error(CMM_ERR_ARG, "batched: plan was not prepared");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(bp.ws);
    cudaError_t e = cudaMemsetAsync(base + bp.off_ctr, 0, bp.ctr_bytes, s);
    if (e != cudaSuccess) return set_error(CMM_ERR_CUDA, cudaGetErrorString(e));
    switch (bp.d) {
        case 3: e = launch_batched_inst<3>(bp, budget_ns, extra, s); break;
        case 5: e = launch_batched_inst<5>(bp, budget_ns, extra, s); break;
        case 7: e = launch_batched_inst<7>(bp, budget_ns, extra, s); break;
        case 9: e = launch_batched_inst<9>(bp, budget_ns, extra, s); break;
        default: e = launch_batched_inst<0>(bp, budget_ns, extra, s); break;
    }
    if (e != cudaSuccess) return set_error(CMM_ERR_CUDA, cudaGetErrorString(e));
    return CMM_OK;
}

extern "C" int cmm_batched_status(const cmm_batch_plan *plan, void *stream) {
    if (!plan) return set_error(CMM_ERR_ARG, "batched: plan is NULL");
    BPlan bp;
    std::memcpy(&bp, plan, sizeof bp);
    if (bp.magic != kPlanMagic) return set_error(CMM_ERR_ARG, "batched: plan was not prepared");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int err = 0;
    cudaError_t e = cudaMemcpyAsync(&err, static_cast<char *>(bp.ws) + bp.off_ctr + sizeof(int),
                                    sizeof err, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(CMM_ERR_CUDA, cudaGetErrorString(e));
    if (err) return set_error(CMM_ERR_TIMEOUT, "batched: a bounded dependency wait ran out");
    return CMM_OK;
}
