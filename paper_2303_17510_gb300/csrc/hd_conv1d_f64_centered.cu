// Fused 1D convolution kernels: f64, centered data (instantiation unit).
#define HD_REAL double
#define HD_KIND hd::KIND_CENTERED
#define HD_DT f64
#define HD_KN centered
#define HD_VARIANTS(X) X(2, 2, 1) X(4, 4, 1) X(8, 8, 1) X(16, 8, 1) X(32, 8, 1) X(64, 8, 1) X(128, 8, 1) X(256, 8, 1) X(512, 8, 1) X(1024, 8, 1) X(2048, 8, 1)
#include "hd_conv1d_tu.cuh"
