// Split-path kernels (transforms larger than one CTA), FP32.
#define HD_REAL float
#define HD_DT f32
#define HD_S2 4096
#include "hd_split_tu.cuh"
