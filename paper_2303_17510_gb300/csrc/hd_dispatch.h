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
    bool comp;   // compensated (TwoSum) accumulation of residue contributions
    int minb;    // CTAs per SM the register allocation allows (1 or 2)
};

// dynamic shared memory limit of one CTA on sm_103a
constexpr size_t kMaxSmemPerBlock = 227 * 1024;

// true when a kernel instance exists for cfg and its shared memory fits for
// staged rows of ls_pad values
bool conv1d_available(const Conv1dCfg& c, int ls_pad);
// launch `count` convolutions (a.count) of cfg on stream
cudaError_t conv1d_launch(const Conv1dCfg& c, const ConvArgs& a, cudaStream_t st);
// cluster variant (D residue groups per convolution, D > 1): available for
// cfg (S, E, kind, mult, nb) with rows of ls_pad values, and its launch
bool conv1d_cluster_available(const Conv1dCfg& c, int ls_pad, int D);
cudaError_t conv1d_cluster_launch(const Conv1dCfg& c, const ConvArgs& a, int D, cudaStream_t st);
// compiled (S, E, minb) variants for cfg's dtype and kind; returns the count
int conv1d_variants(int dtype, int kind, Conv1dCfg* out, int cap);
// forward transform of residue r of one input (debug path)
cudaError_t forward_residue_launch(const Conv1dCfg& c, const ConvArgs& a, int r, int m, void* out, cudaStream_t st);

struct SplitArgs;
// split path: colfwd / row / colbwd kernels for one chunk of instances
cudaError_t split_launch_f32(const SplitArgs& a, int kind, int mult, bool comp, cudaStream_t st);
cudaError_t split_launch_f64(const SplitArgs& a, int kind, int mult, bool comp, cudaStream_t st);

struct ColArgs;
// outer-axis column kernels (forward or backward) for one residue block
cudaError_t col_launch_f32(const ColArgs& a, int kind, bool comp, bool fwd, cudaStream_t st);
cudaError_t col_launch_f64(const ColArgs& a, int kind, bool comp, bool fwd, cudaStream_t st);
// values per thread of the column FFT of size S (its twiddle table layout)
int col_E_of_f32(int S);
int col_E_of_f64(int S);

// per translation unit entry points (dtype x kind x mult set: the
// single-output mults, the two-output one in the _b2 units, the five-output
// one in the _b5 units, the eight-output one in the _b8 units)
#define HD_DECL_TU(DT, KN)                                                                                   \
    bool conv1d_available_##DT##_##KN(const Conv1dCfg& c, int ls_pad);                                                    \
    cudaError_t conv1d_launch_##DT##_##KN(const Conv1dCfg& c, const ConvArgs& a, cudaStream_t st);            \
    cudaError_t forward_residue_launch_##DT##_##KN(const Conv1dCfg& c, const ConvArgs& a, int r, int m,       \
                                                    void* out, cudaStream_t st);                              \
    int conv1d_variants_##DT##_##KN(Conv1dCfg* out, int cap);                                                \
    bool conv1d_cluster_available_##DT##_##KN(const Conv1dCfg& c, int ls_pad, int D);                          \
    cudaError_t conv1d_cluster_launch_##DT##_##KN(const Conv1dCfg& c, const ConvArgs& a, int D, cudaStream_t st); \
    int conv1d_take_error_##DT##_##KN();
HD_DECL_TU(f32, complex)
HD_DECL_TU(f32, centered)
HD_DECL_TU(f32, hermitian)
HD_DECL_TU(f64, complex)
HD_DECL_TU(f64, centered)
HD_DECL_TU(f64, hermitian)
HD_DECL_TU(f32, complex_b2)
HD_DECL_TU(f32, centered_b2)
HD_DECL_TU(f32, hermitian_b2)
HD_DECL_TU(f64, complex_b2)
HD_DECL_TU(f64, centered_b2)
HD_DECL_TU(f64, hermitian_b2)
HD_DECL_TU(f32, complex_b5)
HD_DECL_TU(f32, centered_b5)
HD_DECL_TU(f32, hermitian_b5)
HD_DECL_TU(f64, complex_b5)
HD_DECL_TU(f64, centered_b5)
HD_DECL_TU(f64, hermitian_b5)
HD_DECL_TU(f32, complex_b8)
HD_DECL_TU(f32, centered_b8)
HD_DECL_TU(f32, hermitian_b8)
HD_DECL_TU(f64, complex_b8)
HD_DECL_TU(f64, centered_b8)
HD_DECL_TU(f64, hermitian_b8)
#undef HD_DECL_TU

}  // namespace hd
