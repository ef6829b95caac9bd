// sketch_f64.cu -- FP64-butterfly instantiations of the fused sketch kernel.
#include "sketch_impl.cuh"

namespace cmm {

namespace {
template <int L>
struct F64Cfg {
    static constexpr int LE = L < 4 ? L : 4;
    static constexpr int THREADS = L == 13 ? 512 : 256;
};

template <int L>
cudaError_t run(const SketchPlan &pl, const double *At, const double *Bp, int64_t m, int64_t k,
                int64_t p, int d, const HashParams &hp, const tab_t *tabA,
                const tab_t *tabB, const float *colmax, double *partial, cudaStream_t s) {
    return launch_sketch_inst<double, double, L, F64Cfg<L>::LE, F64Cfg<L>::THREADS>(
        pl, At, Bp, m, k, p, d, hp, tabA, tabB, colmax, partial, s);
}

template <int L>
constexpr size_t smem_of() {
    return sketch_smem_bytes<L, F64Cfg<L>::LE, F64Cfg<L>::THREADS, double>();
}
}  // namespace

int sketch_threads_f64(int Llo) {
    switch (Llo) {
#define CASE(L) case L: return F64Cfg<L>::THREADS;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10)
        CASE(11) CASE(12) CASE(13)
#undef CASE
    }
    return 0;
}

size_t sketch_smem_f64(int Llo) {
    switch (Llo) {
#define CASE(L) case L: return smem_of<L>();
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10)
        CASE(11) CASE(12) CASE(13)
#undef CASE
    }
    return 0;
}

cudaError_t launch_sketch_f64(const SketchPlan &pl, const double *At, const double *Bp, int64_t m,
                              int64_t k, int64_t p, int d, const HashParams &hp,
                              const tab_t *tabA, const tab_t *tabB, const float *colmax,
                              double *partial, cudaStream_t s) {
    switch (pl.Llo) {
#define CASE(L) case L: return run<L>(pl, At, Bp, m, k, p, d, hp, tabA, tabB, colmax, partial, s);
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10)
        CASE(11) CASE(12) CASE(13)
#undef CASE
    }
    return cudaErrorInvalidValue;
}

}  // namespace cmm
