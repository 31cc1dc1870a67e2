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

// Five-output mult (3D Basdevant): one variant per size, one CTA per SM (the
// residue sums of the five outputs live in shared memory).
#define HD_VARIANTS_F32_B5(X) \
    X(2, 2, 1) X(4, 4, 1) X(8, 8, 1) X(16, 8, 1) X(32, 8, 1) X(64, 8, 1) X(128, 8, 1) X(256, 8, 1) X(512, 8, 1) \
    X(1024, 8, 1) X(2048, 8, 1)
#define HD_VARIANTS_F64_B5(X) \
    X(2, 2, 1) X(4, 4, 1) X(8, 8, 1) X(16, 8, 1) X(32, 8, 1) X(64, 8, 1) X(128, 8, 1) X(256, 8, 1) X(512, 8, 1) \
    X(1024, 8, 1)

// Eight-output mult (3D MHD, six inputs): one variant per size, one CTA per SM;
// the residue sums of the eight outputs live in shared memory (16 S values),
// which leaves FP32 transforms of 1024 points and FP64 of 512 to short rows.
#define HD_VARIANTS_F32_B8(X) \
    X(2, 2, 1) X(4, 4, 1) X(8, 8, 1) X(16, 8, 1) X(32, 8, 1) X(64, 8, 1) X(128, 8, 1) X(256, 8, 1) X(512, 8, 1) \
    X(1024, 8, 1)
#define HD_VARIANTS_F64_B8(X) \
    X(2, 2, 1) X(4, 4, 1) X(8, 8, 1) X(16, 8, 1) X(32, 8, 1) X(64, 8, 1) X(128, 8, 1) X(256, 8, 1) X(512, 8, 1)

// Cluster variants (D > 1 residues per pass, one convolution per cluster), as X(S, E).
// FP64 takes E = 4 and 2 as well: a CTA of S/4 or S/2 threads spreads over all
// four SM sub-partitions (each with its own FP64 unit) with more warps to
// cover the FP64 latency.
#define HD_CLUSTER_VARIANTS_F32(X) X(256, 8) X(512, 8) X(1024, 8) X(2048, 8) X(4096, 8)
#define HD_CLUSTER_VARIANTS_F64(X) \
    X(256, 8) X(512, 8) X(1024, 8) X(2048, 8) X(256, 4) X(512, 4) X(1024, 4) X(256, 2) X(512, 2)

#define HD_VARIANTS_F64(X) \
    X(2, 2, 1) X(4, 4, 1) X(8, 8, 1) X(16, 8, 1) X(32, 8, 1) X(64, 8, 1) X(128, 8, 1) X(256, 8, 1) \
    X(512, 8, 1) X(1024, 8, 1) X(2048, 8, 1)
