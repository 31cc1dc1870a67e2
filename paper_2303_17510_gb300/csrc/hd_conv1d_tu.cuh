// hd_conv1d_tu.cuh -- instantiation table of the fused 1D kernels for one
// (dtype, kind) pair.  Included by the hd_conv1d_<dtype>_<kind>.cu files with
// HD_REAL, HD_KIND, HD_DT and HD_KN defined.
#include "hd_dispatch.h"

namespace hd {

namespace {

template <class R, int S, int E, int KIND, int MULT, int NB>
cudaError_t launch_one(const ConvArgs& a, cudaStream_t st) {
    constexpr int T = S / E;
    constexpr int G = (256 / T) < 1 ? 1 : (256 / T);
    const size_t smem = size_t(G) * FftShape<S, E>::SMEM * sizeof(cplx<R>);
    auto k = conv1d_kernel<R, S, E, KIND, MULT, NB, G>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t blocks = (a.count + G - 1) / G;
    if (blocks <= 0) return cudaSuccess;
    k<<<dim3((unsigned)blocks), dim3(G * T), smem, st>>>(a);
    return cudaGetLastError();
}

template <class R, int S, int E, int KIND>
cudaError_t launch_fwd(const ConvArgs& a, int r, int m, void* out, cudaStream_t st) {
    const size_t smem = FftShape<S, E>::SMEM * sizeof(cplx<R>);
    auto k = forward_residue_kernel<R, S, E, KIND>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<1, S / E, smem, st>>>(a, r, m, out);
    return cudaGetLastError();
}

}  // namespace

// (S, E) pairs compiled for this dtype: every power of two up to HD_SMAX with
// E = 8 (E = S below 8), plus E = 16 where registers allow (one folded block,
// product mult, FP32).
#define HD_SE_LIST(X)                                                                                        \
    X(2, 2) X(4, 4) X(8, 8) X(16, 8) X(32, 8) X(64, 8) X(128, 8) X(256, 8) X(512, 8) X(1024, 8) X(2048, 8)   \
    HD_SE_EXTRA(X)

// Combinations that get a kernel: Hermitian data folds into one output block,
// centered data into two; E = 16 keeps 2E accumulators plus three spectra in
// registers only for one block and the binary product.
template <int E, int MULT, int NB>
constexpr bool combo_ok() {
    return !((HD_KIND == KIND_HERMITIAN && NB != 1) || (HD_KIND == KIND_CENTERED && NB != 2) ||
             (E == 16 && (NB != 1 || MULT != MULT_PRODUCT)));
}

template <int S, int E, int MULT, int NB>
cudaError_t pick(const ConvArgs& a, cudaStream_t st) {
    if constexpr (combo_ok<E, MULT, NB>()) return launch_one<HD_REAL, S, E, HD_KIND, MULT, NB>(a, st);
    else return cudaErrorInvalidValue;
}

#define HD_NBMULT_CASES(SS, EE)                                                                                \
    if (c.S == SS && c.E == EE) {                                                                              \
        if (c.mult == MULT_PRODUCT && c.nb == 1) return pick<SS, EE, MULT_PRODUCT, 1>(a, st);                  \
        if (c.mult == MULT_PAIRS3 && c.nb == 1) return pick<SS, EE, MULT_PAIRS3, 1>(a, st);                    \
        if (c.mult == MULT_PRODUCT && c.nb == 2) return pick<SS, EE, MULT_PRODUCT, 2>(a, st);                  \
        if (c.mult == MULT_PAIRS3 && c.nb == 2) return pick<SS, EE, MULT_PAIRS3, 2>(a, st);                    \
    }

#define HD_AVAIL_CASE(SS, EE)                                                                                  \
    if (c.S == SS && c.E == EE) {                                                                              \
        if (c.mult == MULT_PRODUCT && c.nb == 1) return combo_ok<EE, MULT_PRODUCT, 1>();                      \
        if (c.mult == MULT_PAIRS3 && c.nb == 1) return combo_ok<EE, MULT_PAIRS3, 1>();                        \
        if (c.mult == MULT_PRODUCT && c.nb == 2) return combo_ok<EE, MULT_PRODUCT, 2>();                      \
        if (c.mult == MULT_PAIRS3 && c.nb == 2) return combo_ok<EE, MULT_PAIRS3, 2>();                        \
        return false;                                                                                        \
    }
#define HD_FWD_CASE(SS, EE) if (c.S == SS && c.E == EE) return launch_fwd<HD_REAL, SS, EE, HD_KIND>(a, r, m, out, st);

#define HD_CAT2(a, b, c, d) a##b##c##d
#define HD_FN(base, DT, KN) HD_CAT2(base, DT, _, KN)

bool HD_FN(conv1d_available_, HD_DT, HD_KN)(const Conv1dCfg& c) {
    HD_SE_LIST(HD_AVAIL_CASE)
    return false;
}

cudaError_t HD_FN(conv1d_launch_, HD_DT, HD_KN)(const Conv1dCfg& c, const ConvArgs& a, cudaStream_t st) {
    HD_SE_LIST(HD_NBMULT_CASES)
    return cudaErrorInvalidValue;
}

cudaError_t HD_FN(forward_residue_launch_, HD_DT, HD_KN)(const Conv1dCfg& c, const ConvArgs& a, int r, int m,
                                                         void* out, cudaStream_t st) {
    HD_SE_LIST(HD_FWD_CASE)
    return cudaErrorInvalidValue;
}

}  // namespace hd
