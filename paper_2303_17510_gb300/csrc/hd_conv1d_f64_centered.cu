// Fused 1D convolution kernels: f64, centered data (instantiation unit).
#define HD_REAL double
#define HD_KIND hd::KIND_CENTERED
#define HD_DT f64
#define HD_KN centered
#define HD_SE_EXTRA(X) 
#include "hd_conv1d_tu.cuh"
