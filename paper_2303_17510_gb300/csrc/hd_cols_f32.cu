// Outer-axis column kernels of multidimensional convolutions, FP32.
#define HD_REAL float
#define HD_DT f32
#define HD_SMAX 4096
#include "hd_cols_tu.cuh"
