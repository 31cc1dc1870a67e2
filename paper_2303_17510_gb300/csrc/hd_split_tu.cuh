// hd_split_tu.cuh -- instantiations and launcher of the split path for one
// dtype (HD_REAL, HD_DT, HD_S2 defined by the including unit).
#include "hd_dispatch.h"
#include "hd_split.cuh"

namespace hd {

namespace {

template <int S1, int KIND, int MULT, bool COMP>
cudaError_t run_split(const SplitArgs& a, cudaStream_t st) {
    using R = HD_REAL;
    constexpr int S2 = HD_S2;
    constexpr int E = 8;
    constexpr int T = S2 / E;
    constexpr int NX = MultShape<MULT>::NX;
    const int64_t n1 = a.count * a.A * a.nr * (int64_t)S2;
    if (n1 <= 0) return cudaSuccess;
    split_colfwd<R, S1, KIND><<<(unsigned)((n1 + 255) / 256), 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int G = (256 / T) < 1 ? 1 : 256 / T;
    const size_t smem = size_t(G) * NX * FftShape<S2, E>::SMEM * sizeof(cplx<R>);
    auto rk = split_row<R, S2, E, KIND == KIND_HERMITIAN ? KIND_HERMITIAN : KIND_COMPLEX, MULT>;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(rk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t rows = a.count * a.nr * (int64_t)S1;
    rk<<<(unsigned)((rows + G - 1) / G), G * T, smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t n3 = a.count * a.B * (int64_t)S2;
    split_colbwd<R, S1, KIND, COMP><<<(unsigned)((n3 + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <int S1, int KIND, int MULT>
cudaError_t by_comp(const SplitArgs& a, bool comp, cudaStream_t st) {
    constexpr bool F64 = sizeof(HD_REAL) == 8;
    if (comp && !F64) return run_split<S1, KIND, MULT, true>(a, st);
    return run_split<S1, KIND, MULT, false>(a, st);
}

template <int S1, int KIND>
cudaError_t by_mult(const SplitArgs& a, int mult, bool comp, cudaStream_t st) {
    switch (mult) {
        case MULT_PRODUCT: return by_comp<S1, KIND, MULT_PRODUCT>(a, comp, st);
        case MULT_PAIRS3: return by_comp<S1, KIND, MULT_PAIRS3>(a, comp, st);
        case MULT_BASD2: return by_comp<S1, KIND, MULT_BASD2>(a, comp, st);
        case MULT_BASD3: return by_comp<S1, KIND, MULT_BASD3>(a, comp, st);
        case MULT_MHD3: return by_comp<S1, KIND, MULT_MHD3>(a, comp, st);
    }
    return cudaErrorInvalidValue;
}

template <int S1>
cudaError_t by_kind(const SplitArgs& a, int kind, int mult, bool comp, cudaStream_t st) {
    if (kind == KIND_COMPLEX) return by_mult<S1, KIND_COMPLEX>(a, mult, comp, st);
    if (kind == KIND_CENTERED) return by_mult<S1, KIND_CENTERED>(a, mult, comp, st);
    return by_mult<S1, KIND_HERMITIAN>(a, mult, comp, st);
}

}  // namespace

#define HD_CAT3(a, b) a##b
#define HD_FN2(base, DT) HD_CAT3(base, DT)

cudaError_t HD_FN2(split_launch_, HD_DT)(const SplitArgs& a, int kind, int mult, bool comp, cudaStream_t st) {
    switch (a.S1) {
        case 2: return by_kind<2>(a, kind, mult, comp, st);
        case 4: return by_kind<4>(a, kind, mult, comp, st);
        case 8: return by_kind<8>(a, kind, mult, comp, st);
        case 16: return by_kind<16>(a, kind, mult, comp, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace hd
