// Fused 1D convolution kernels: f64, centered data, the single-output mults (instantiation unit).
#define HD_REAL double
#define HD_KIND hd::KIND_CENTERED
#define HD_DT f64
#define HD_KN centered
#define HD_VARIANTS HD_VARIANTS_F64
#define HD_CLUSTER_VARIANTS HD_CLUSTER_VARIANTS_F64
#define HD_UNIT_MULTS(Y, ...) Y(MULT_PRODUCT, __VA_ARGS__) Y(MULT_PAIRS3, __VA_ARGS__)
#include "hd_conv1d_variants.h"
#include "hd_conv1d_tu.cuh"
