// hd_cols.cuh -- residue transforms along an outer axis of a multidimensional
// convolution (Section 5: an n-D convolution is the padded FFTs along the first
// axis, lower-dimensional sub-convolutions, and the inverse FFTs along the
// first axis; Fig. conv2psimp4 for the 2D memory reuse).
//
// A CTA handles a tile of TY adjacent columns (the elements that share every
// inner index) and one residue of one input: thread (tau, y) with y fastest,
// so every global load and store moves whole 32-byte sectors of TY columns.
// The columns' size-S FFTs run in shared memory interleaved column by column
// (CST = TY), which keeps the exchanges free of bank conflicts.
//
// Work buffer layout: F[a][inst][r'][slot][col] (a < max(A, B): the inner
// sub-convolutions write output b over input b), slot = tau + T e labels the
// spectral value held in register e (any fixed labeling of the outer
// frequencies works: the inner sub-convolution treats every slot row
// independently).  For each outer instance the rows F[a][inst][r'][slot][:] are
// contiguous inner sub-arrays, so the inner axes are a plain batch.
#pragma once

#include "hd_conv1d.cuh"

namespace hd {

struct ColArgs {
    const void* f[kMaxIn];   // colfwd: A input bases; element (inst, x, col) at f + inst*inst_stride + x*pitch + col
    void* work;           // F[a][inst][r'][slot][col]
    void* h[kMaxOut];     // colbwd: B output bases, same layout as the inputs
    int64_t inst_stride;  // elements between outer instances
    int64_t count;        // outer instances
    int64_t pitch;        // elements between consecutive x of one column
    int64_t ncols;        // columns per instance
    int L, H;             // stored axis length, centered offset floor(L/2)
    int n, S, A, B;       // residues of the axis, transform size, inputs, outputs
    int r0, nr;           // residue block handled by this call
    int accumulate;       // colbwd: add to h (blocks after the first)
    const void* twS;      // FFT pass twiddles of (S, E)
    const void* twN;      // residue twists [r][j], then zeta_N^{r S}
    double invN;          // 1 / (q m) of the axis
};

template <int S, int E>
struct ColShape {
    static constexpr int T = S / E;
    static constexpr int TY = (512 / T) > 32 ? 32 : ((512 / T) < 1 ? 1 : 512 / T);
    static constexpr int THREADS = T * TY;
};

// Forward: input blockIdx.y, all nr residues of the block: the column tile is
// read once (both folded blocks kept in registers), then per residue fold +
// twist, FFT along x, spectral values to the work buffer.  Residue 0 (r0 = 0)
// has unit twists.  Tiles of 256 threads (S <= 128) are held to two CTAs per
// SM (128 registers, no spills): left alone the compiler took 164 registers,
// one CTA per SM, and the 256^3 Hermitian plan ran 10 % slower.
template <class R, int S, int E, int KIND>
__global__ void __launch_bounds__(ColShape<S, E>::THREADS, ColShape<S, E>::THREADS <= 256 ? 2 : 1)
    col_forward(const __grid_constant__ ColArgs a) {
    using T = cplx<R>;
    using CS = ColShape<S, E>;
    constexpr int TY = CS::TY;
    constexpr int TT = CS::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int y = threadIdx.x % TY;
    const int tau = threadIdx.x / TY;
    const int64_t col = (int64_t)blockIdx.x * TY + y;
    const bool valid = col < a.ncols;
    const int aa = blockIdx.y;
    const int64_t inst = blockIdx.z;
    T* sm = reinterpret_cast<T*>(smem_raw) + y;
    const TwGlobalProducts<T> tw{static_cast<const T*>(a.twS)};
    const T* twN = static_cast<const T*>(a.twN);
    const T* f = static_cast<const T*>(a.f[aa]) + inst * a.inst_stride + (valid ? col : 0);
    T b0[E], b1[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int j = tau + TT * e;
        b0[e] = czero<T>();
        b1[e] = czero<T>();
        if (valid) {
            // read once: streaming loads, so the column data does not evict the
            // twiddle tables from L1
            if constexpr (KIND == KIND_COMPLEX) {
                if (j < a.L) b0[e] = ld_in<true>(f, (int64_t)j * a.pitch);
                if (j + S < a.L) b1[e] = ld_in<true>(f, (int64_t)(j + S) * a.pitch);
            } else {
                if (j < a.L - a.H) b0[e] = ld_in<true>(f, (int64_t)(j + a.H) * a.pitch);
                if (j >= S - a.H) b1[e] = ld_in<true>(f, (int64_t)(j - S + a.H) * a.pitch);
            }
        }
    }
    for (int rr = 0; rr < a.nr; ++rr) {
        const int r = a.r0 + rr;
        T v[E];
        if (r == 0) {
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = cadd(b0[e], b1[e]);
        } else {
            T cr = ldtw(twN + (int64_t)a.n * S + r);
            if constexpr (KIND == KIND_CENTERED) cr = cconj(cr);
            const TwistRow tr = twist_row(r, a.n);   // conjugate symmetry
#pragma unroll
            for (int e = 0; e < E; ++e)
                v[e] = cmul(cadd(b0[e], cmul(cr, b1[e])), twist_ld(twN + (int64_t)tr.row * S + tau + TT * e, tr.conj));
        }
        fft_forward<S, E, 1, TY>(v, sm, tw, tau);
        if (valid) {
            T* w = static_cast<T*>(a.work) + (((int64_t)aa * a.count + inst) * a.nr + rr) * (int64_t)S * a.ncols + col;
#pragma unroll
            for (int e = 0; e < E; ++e) w[(int64_t)(tau + TT * e) * a.ncols] = v[e];
        }
    }
}

// Backward: output blockIdx.y; for every residue of the block, inverse FFT
// along x of the sub-convolution results (held in part b of the work buffer),
// the conjugate twist, and the residue sum; one store (or add) per output.
template <class R, int S, int E, int KIND, bool COMP>
__global__ void __launch_bounds__(ColShape<S, E>::THREADS) col_backward(const __grid_constant__ ColArgs a) {
    using T = cplx<R>;
    using CS = ColShape<S, E>;
    constexpr int TY = CS::TY;
    constexpr int TT = CS::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int y = threadIdx.x % TY;
    const int tau = threadIdx.x / TY;
    const int64_t col = (int64_t)blockIdx.x * TY + y;
    const bool valid = col < a.ncols;
    const int ob = blockIdx.y;
    const int64_t inst = blockIdx.z;
    T* sm = reinterpret_cast<T*>(smem_raw) + y;
    const TwGlobalProducts<T> tw{static_cast<const T*>(a.twS)};
    const T* twN = static_cast<const T*>(a.twN);
    R s0[2 * E], c0[COMP ? 2 * E : 1], s1[2 * E], c1[COMP ? 2 * E : 1];
    R dummy = 0;
#pragma unroll
    for (int i = 0; i < 2 * E; ++i) {
        s0[i] = s1[i] = 0;
        if constexpr (COMP) c0[i] = c1[i] = 0;
    }
    for (int rr = 0; rr < a.nr; ++rr) {
        const int r = a.r0 + rr;
        T cr = ldtw(twN + (int64_t)a.n * S + r);
        if constexpr (KIND == KIND_CENTERED) cr = cconj(cr);
        const T* g = static_cast<const T*>(a.work) + (((int64_t)ob * a.count + inst) * a.nr + rr) * (int64_t)S * a.ncols +
                     (valid ? col : 0);
        T v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = valid ? ld_in<true>(g, (int64_t)(tau + TT * e) * a.ncols) : czero<T>();
        fft_inverse<S, E, 1, TY>(v, sm, tw, tau);
        const bool r0 = r == 0;   // unit twists
        const TwistRow tr = twist_row(r, a.n);   // conjugate symmetry
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int j = tau + TT * e;
            const T yv = r0 ? v[e] : cmulc(v[e], twist_ld(twN + (int64_t)tr.row * S + j, tr.conj));
            acc_add<R, COMP>(s0[2 * e], COMP ? c0[2 * e] : dummy, yv.x);
            acc_add<R, COMP>(s0[2 * e + 1], COMP ? c0[2 * e + 1] : dummy, yv.y);
            const T y1 = r0 ? yv : cmulc(yv, cr);
            acc_add<R, COMP>(s1[2 * e], COMP ? c1[2 * e] : dummy, y1.x);
            acc_add<R, COMP>(s1[2 * e + 1], COMP ? c1[2 * e + 1] : dummy, y1.y);
        }
    }
    if (!valid) return;
    T* hout = static_cast<T*>(a.h[ob]) + inst * a.inst_stride + col;
    const R sc = R(a.invN);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int j = tau + TT * e;
        const R x0 = COMP ? s0[2 * e] + c0[2 * e] : s0[2 * e];
        const R y0 = COMP ? s0[2 * e + 1] + c0[2 * e + 1] : s0[2 * e + 1];
        const R x1 = COMP ? s1[2 * e] + c1[2 * e] : s1[2 * e];
        const R y1 = COMP ? s1[2 * e + 1] + c1[2 * e + 1] : s1[2 * e + 1];
        const T o0 = mk<T>(x0 * sc, y0 * sc), o1 = mk<T>(x1 * sc, y1 * sc);
        int x0i = -1, x1i = -1;
        if constexpr (KIND == KIND_COMPLEX) {
            if (j < a.L) x0i = j;
            if (j + S < a.L) x1i = j + S;
        } else {
            if (j < a.L - a.H) x0i = j + a.H;
            if (j >= S - a.H) x1i = j - S + a.H;
        }
        if (x0i >= 0) {
            T* p = hout + (int64_t)x0i * a.pitch;
            *p = a.accumulate ? cadd(*p, o0) : o0;
        }
        if (x1i >= 0) {
            T* p = hout + (int64_t)x1i * a.pitch;
            *p = a.accumulate ? cadd(*p, o1) : o1;
        }
    }
}

}  // namespace hd
