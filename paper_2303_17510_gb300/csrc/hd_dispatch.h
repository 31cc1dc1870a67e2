// hd_dispatch.h -- host-side launch interface of the fused 1D kernels.
#pragma once

#include <cuda_runtime.h>

#include "hd_conv1d.cuh"

namespace hd {

struct Conv1dCfg {
    int dtype;   // 0 f32, 1 f64
    int kind;    // KIND_*
    int mult;    // MULT_*
    int nb;      // folded blocks: 1 or 2
    int S;       // transform size (power of two)
    int E;       // values per thread
};

// Groups (convolutions) per CTA for a transform of size S with E values per thread.
inline int conv1d_groups(int S, int E) {
    int T = S / E;
    int G = 256 / T;
    return G < 1 ? 1 : G;
}

// true when a kernel instance exists for cfg
bool conv1d_available(const Conv1dCfg& c);
// launch `count` convolutions (a.count) of cfg on stream
cudaError_t conv1d_launch(const Conv1dCfg& c, const ConvArgs& a, cudaStream_t st);
// forward transform of residue r of one input (debug path)
cudaError_t forward_residue_launch(const Conv1dCfg& c, const ConvArgs& a, int r, int m, void* out, cudaStream_t st);

// per translation unit entry points (dtype x kind)
#define HD_DECL_TU(DT, KN)                                                                                   \
    bool conv1d_available_##DT##_##KN(const Conv1dCfg& c);                                                    \
    cudaError_t conv1d_launch_##DT##_##KN(const Conv1dCfg& c, const ConvArgs& a, cudaStream_t st);            \
    cudaError_t forward_residue_launch_##DT##_##KN(const Conv1dCfg& c, const ConvArgs& a, int r, int m,       \
                                                    void* out, cudaStream_t st);
HD_DECL_TU(f32, complex)
HD_DECL_TU(f32, centered)
HD_DECL_TU(f32, hermitian)
HD_DECL_TU(f64, complex)
HD_DECL_TU(f64, centered)
HD_DECL_TU(f64, hermitian)
#undef HD_DECL_TU

}  // namespace hd
