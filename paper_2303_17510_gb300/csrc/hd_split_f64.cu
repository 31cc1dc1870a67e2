// Split-path kernels (transforms larger than one CTA), FP64.
#define HD_REAL double
#define HD_DT f64
#define HD_S2 2048
#include "hd_split_tu.cuh"
