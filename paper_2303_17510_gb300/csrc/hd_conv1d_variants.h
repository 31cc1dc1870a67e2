// hd_conv1d_variants.h -- (S, E, MINB) variants of the fused 1D kernels that
// every instantiation unit of a dtype compiles (X(S, E, MINB) per variant).
// FP32: 2 CTAs per SM (at most 128 registers) up to S = 2048, one CTA per SM
// with E = 4, 8, 16 for the larger transforms; FP64: one CTA per SM.
#pragma once

#define HD_VARIANTS_F32(X) \
    X(2, 2, 2) X(4, 4, 2) X(8, 8, 2) X(16, 8, 2) X(32, 8, 2) X(64, 8, 2) X(128, 8, 2) X(256, 8, 2) \
    X(512, 8, 2) X(1024, 8, 2) X(2048, 8, 2) X(4096, 8, 1) X(512, 8, 1) X(1024, 8, 1) X(2048, 8, 1) \
    X(512, 4, 1) X(1024, 4, 1) X(2048, 4, 1) X(256, 16, 1) X(512, 16, 1) X(1024, 16, 1) \
    X(2048, 16, 1) X(4096, 16, 1)

#define HD_VARIANTS_F64(X) \
    X(2, 2, 1) X(4, 4, 1) X(8, 8, 1) X(16, 8, 1) X(32, 8, 1) X(64, 8, 1) X(128, 8, 1) X(256, 8, 1) \
    X(512, 8, 1) X(1024, 8, 1) X(2048, 8, 1)
