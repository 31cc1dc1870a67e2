// Fused 1D convolution kernels: f64, hermitian data, the eight-output mult (3D MHD) (instantiation unit).
#define HD_REAL double
#define HD_KIND hd::KIND_HERMITIAN
#define HD_DT f64
#define HD_KN hermitian_b8
#define HD_VARIANTS HD_VARIANTS_F64_B8
#define HD_CLUSTER_VARIANTS HD_CLUSTER_VARIANTS_F64
#define HD_UNIT_MULTS(Y, ...) Y(MULT_MHD3, __VA_ARGS__)
#include "hd_conv1d_variants.h"
#include "hd_conv1d_tu.cuh"
