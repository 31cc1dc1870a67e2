// Fused 1D convolution kernels: f32, centered data (instantiation unit).
#define HD_REAL float
#define HD_KIND hd::KIND_CENTERED
#define HD_DT f32
#define HD_KN centered
#define HD_SE_EXTRA(X) X(4096, 8)
#include "hd_conv1d_tu.cuh"
