// Outer-axis column kernels of multidimensional convolutions, FP64.
#define HD_REAL double
#define HD_DT f64
#define HD_SMAX 2048
#include "hd_cols_tu.cuh"
