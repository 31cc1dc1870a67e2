// Fused 1D convolution kernels: f32, centered data (instantiation unit).
#define HD_REAL float
#define HD_KIND hd::KIND_CENTERED
#define HD_DT f32
#define HD_KN centered
#define HD_VARIANTS(X) X(2, 2, 2) X(4, 4, 2) X(8, 8, 2) X(16, 8, 2) X(32, 8, 2) X(64, 8, 2) X(128, 8, 2) X(256, 8, 2) X(512, 8, 2) X(1024, 8, 2) X(2048, 8, 2) X(4096, 8, 1) X(512, 8, 1) X(1024, 8, 1) X(2048, 8, 1) X(512, 4, 1) X(1024, 4, 1) X(2048, 4, 1) X(256, 16, 1) X(512, 16, 1) X(1024, 16, 1) X(2048, 16, 1) X(4096, 16, 1)
#include "hd_conv1d_tu.cuh"
