// hd_cols_tu.cuh -- instantiations and launchers of the outer-axis column
// kernels for one dtype (HD_REAL, HD_DT, HD_SMAX defined by the includer).
#include "hd_cols.cuh"
#include "hd_dispatch.h"

namespace hd {

namespace {

// values per thread of the column FFT: 16 from S = 128 on (two passes at S = 128
// instead of the three of E = 8: 6 % faster on the 256^3 Hermitian plan, whose
// outer axes take S = 128), else 8 (or S below 8)
template <int S>
constexpr int col_E() {
    return S < 128 ? (S < 8 ? S : 8) : 16;
}

template <int S, int KIND, bool COMP, bool FWD>
cudaError_t col_run(const ColArgs& a, cudaStream_t st) {
    using R = HD_REAL;
    constexpr int E = col_E<S>();
    using CS = ColShape<S, E>;
    const size_t smem = size_t(CS::TY) * FftShape<S, E>::SMEM * sizeof(cplx<R>);
    const unsigned gx = (unsigned)((a.ncols + CS::TY - 1) / CS::TY);
    if (a.count <= 0 || a.ncols <= 0) return cudaSuccess;
    if (a.count > 65535) return cudaErrorInvalidValue;
    if constexpr (FWD) {
        auto k = col_forward<R, S, E, KIND>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k<<<dim3(gx, (unsigned)a.A, (unsigned)a.count), CS::THREADS, smem, st>>>(a);
    } else {
        auto k = col_backward<R, S, E, KIND, COMP>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k<<<dim3(gx, (unsigned)a.B, (unsigned)a.count), CS::THREADS, smem, st>>>(a);
    }
    return cudaGetLastError();
}

// Outer-axis residue sums are plain (compensation is an option of the 1D
// kernels, whose residue sums are longer; here it would spill registers).
template <int S>
cudaError_t col_dispatch(const ColArgs& a, int kind, bool comp, bool fwd, cudaStream_t st) {
    (void)comp;
    if (fwd) return kind == KIND_COMPLEX ? col_run<S, KIND_COMPLEX, false, true>(a, st)
                                         : col_run<S, KIND_CENTERED, false, true>(a, st);
    return kind == KIND_COMPLEX ? col_run<S, KIND_COMPLEX, false, false>(a, st)
                                : col_run<S, KIND_CENTERED, false, false>(a, st);
}

}  // namespace

#define HD_CAT3(a, b) a##b
#define HD_FN2(base, DT) HD_CAT3(base, DT)

cudaError_t HD_FN2(col_launch_, HD_DT)(const ColArgs& a, int kind, bool comp, bool fwd, cudaStream_t st) {
    switch (a.S) {
        case 2: return col_dispatch<2>(a, kind, comp, fwd, st);
        case 4: return col_dispatch<4>(a, kind, comp, fwd, st);
        case 8: return col_dispatch<8>(a, kind, comp, fwd, st);
        case 16: return col_dispatch<16>(a, kind, comp, fwd, st);
        case 32: return col_dispatch<32>(a, kind, comp, fwd, st);
        case 64: return col_dispatch<64>(a, kind, comp, fwd, st);
        case 128: return col_dispatch<128>(a, kind, comp, fwd, st);
        case 256: return col_dispatch<256>(a, kind, comp, fwd, st);
        case 512: return col_dispatch<512>(a, kind, comp, fwd, st);
        case 1024: return col_dispatch<1024>(a, kind, comp, fwd, st);
        case 2048: return col_dispatch<2048>(a, kind, comp, fwd, st);
#if HD_SMAX >= 4096
        case 4096: return col_dispatch<4096>(a, kind, comp, fwd, st);
#endif
    }
    return cudaErrorInvalidValue;
}

int HD_FN2(col_E_of_, HD_DT)(int S) {
    switch (S) {
        case 2: return col_E<2>();
        case 4: return col_E<4>();
        case 8: return col_E<8>();
        case 16: return col_E<16>();
        case 32: return col_E<32>();
        case 64: return col_E<64>();
        case 128: return col_E<128>();
        default: return 16;
    }
}

}  // namespace hd
