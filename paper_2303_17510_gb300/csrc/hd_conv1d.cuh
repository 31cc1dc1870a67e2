// hd_conv1d.cuh -- fused residue-at-a-time 1D convolution kernel (sm_103a).
//
// One thread group (T = S/E threads) computes one whole convolution: for each
// residue it builds the residue's transform input from the stored inputs,
// runs the forward size-S FFT, applies `mult` in registers, runs the inverse
// FFT and accumulates the residue's contribution into registers; the sum is
// scaled by 1/(qm) and stored once (Alg. convolve / convolveX, Section 2.2:
// residue contributions accumulate, so the transformed residues never leave
// the chip).
//
// Residue transform input.  With N = q m = n S the padded transform of the
// input at k = S l' + ... is reorganized so that residue r needs one size-S
// FFT of
//     W_j = zeta_N^{r j} * sum_{i = j mod S} zeta_N^{r (i - j)} f_i,  0 <= j < S,
// the twisted input folded modulo S:
//   complex p <= 2  (S = m):     i in {j, j + m}         (forward1, forward2;
//                                 Eq. forStan with t = 0, 1)
//   complex p  > 2  (S = p m):   i = j (S >= L)          (forwardInner; the size-p
//                                 DFTs along t and the size-m FFTs form one
//                                 size-pm FFT, Section 6.1)
//   centered        (S = p m/2): i in {j, j - S}         (forward2C, Eq. wDef;
//                                 forwardInnerC, Section 6.2, fold factor
//                                 zeta_n^{-v} = zeta_N^{-v S})
//   Hermitian       (S = p m/2): as centered with f_{-c} = conj f_c (Eq. wHerDef)
// and the backward contribution of residue r to h_i is
//     zeta_N^{-r i} * IFFT_S(mult(F))_{i mod S}                (Eq. invStan, invInner)
// (backward1/2, backward2C, backwardInner*).  Hermitian residue spectra are
// real (Section 4), so two residues r1, r2 share one complex FFT:
// FFT(W^{r1} + i W^{r2}) = F^{r1} + i F^{r2}; mult acts on the real and
// imaginary parts separately; the inverse of the product splits back by
// y_j = (Y_j + conj Y_{S-j})/2 and (Y_j - conj Y_{S-j})/(2i).
//
// mult maps the A transformed inputs to B transformed outputs pointwise
// (Section 2); each output has its own inverse transform and residue sum.
//
// FP32 accumulation over residues is compensated (TwoSum) from 8 residues on
// (COMP), plain below; FP64 is plain.
#pragma once

#include <cooperative_groups.h>

#include "hd_fft.cuh"

namespace hd {

enum { KIND_COMPLEX = 0, KIND_CENTERED = 1, KIND_HERMITIAN = 2 };
enum { MULT_PRODUCT = 0, MULT_PAIRS3 = 1, MULT_BASD2 = 2, MULT_BASD3 = 3, MULT_MHD3 = 4 };

// Inputs A and outputs B of each mult; NX exchange buffers.
//   MULT_PRODUCT  A = 2, B = 1:  F1 F2
//   MULT_PAIRS3   A = 3, B = 1:  F1 F2 + F2 F3 + F3 F1
//   MULT_BASD2    A = 2, B = 2:  (F1 F2, F1^2 - F2^2), the nonlinear terms of
//                 2D incompressible Navier-Stokes in Basdevant's form
//                 (velocity components in; Section 9 counts A = B = 2)
//   MULT_BASD3    A = 3, B = 5:  (F1 F2, F2 F3, F3 F1, F1^2 - F3^2, F2^2 - F3^2),
//                 the same for 3D (Section 9 counts A = 3, B = 5)
//   MULT_MHD3     A = 6, B = 8:  inputs the Elsasser components Z+_0..2, Z-_0..2;
//                 outputs the traceless part of T_ij = Z-_i Z+_j: T_01, T_02,
//                 T_10, T_12, T_20, T_21, T_00 - T_22, T_11 - T_22 (3D
//                 incompressible MHD, which Section 9 counts as A = 6, B = 8)
// With B <= 2 the residue sums live in registers and the B inverse
// transforms run together (NX = max(A, B) buffers).  With more outputs
// (OUT_SMEM) the sums live in shared memory, ACC = B * 2 * S values per group
// (each thread owns its own entries), and the inverse transforms run one
// output at a time from the forward spectra kept in registers (NX = A).
template <int MULT>
struct MultShape {
    static constexpr int A = MULT == MULT_MHD3 ? 6 : ((MULT == MULT_PAIRS3 || MULT == MULT_BASD3) ? 3 : 2);
    static constexpr int B = MULT == MULT_BASD2 ? 2 : (MULT == MULT_BASD3 ? 5 : (MULT == MULT_MHD3 ? 8 : 1));
    static constexpr bool OUT_SMEM = B > 2;
    static constexpr int NX = OUT_SMEM ? A : (A > B ? A : B);
    __host__ __device__ static constexpr int acc(int S) { return OUT_SMEM ? B * 2 * S : 0; }
};
constexpr int kMaxOut = 8;
constexpr int kMaxIn = 6;

// arithmetic of mult on complex or real values
__device__ __forceinline__ float xmul(float a, float b) { return a * b; }
__device__ __forceinline__ double xmul(double a, double b) { return a * b; }
__device__ __forceinline__ float2 xmul(float2 a, float2 b) { return cmul(a, b); }
__device__ __forceinline__ double2 xmul(double2 a, double2 b) { return cmul(a, b); }
__device__ __forceinline__ float xadd(float a, float b) { return a + b; }
__device__ __forceinline__ double xadd(double a, double b) { return a + b; }
__device__ __forceinline__ float2 xadd(float2 a, float2 b) { return cadd(a, b); }
__device__ __forceinline__ double2 xadd(double2 a, double2 b) { return cadd(a, b); }
__device__ __forceinline__ float xsub(float a, float b) { return a - b; }
__device__ __forceinline__ double xsub(double a, double b) { return a - b; }
__device__ __forceinline__ float2 xsub(float2 a, float2 b) { return csub(a, b); }
__device__ __forceinline__ double2 xsub(double2 a, double2 b) { return csub(a, b); }

// mult at one point: x[a * XS] (a < A) -> y[b * YS] (b < B).  X is a complex
// value, or a real one for the Hermitian pairs (their spectra are real).
template <int MULT, int XS, int YS, class X>
__device__ __forceinline__ void mult_point(const X* x, X* y) {
    if constexpr (MULT == MULT_PRODUCT) {
        y[0] = xmul(x[0], x[XS]);
    } else if constexpr (MULT == MULT_PAIRS3) {   // F1F2 + F2F3 + F3F1 = F1 F2 + F3 (F1 + F2)
        y[0] = xadd(xmul(x[0], x[XS]), xmul(x[2 * XS], xadd(x[0], x[XS])));
    } else if constexpr (MULT == MULT_BASD2) {     // F1 F2, F1^2 - F2^2 = (F1 + F2)(F1 - F2)
        y[0] = xmul(x[0], x[XS]);
        y[YS] = xmul(xadd(x[0], x[XS]), xsub(x[0], x[XS]));
    } else if constexpr (MULT == MULT_BASD3) {
        y[0] = xmul(x[0], x[XS]);
        y[YS] = xmul(x[XS], x[2 * XS]);
        y[2 * YS] = xmul(x[2 * XS], x[0]);
        y[3 * YS] = xmul(xadd(x[0], x[2 * XS]), xsub(x[0], x[2 * XS]));
        y[4 * YS] = xmul(xadd(x[XS], x[2 * XS]), xsub(x[XS], x[2 * XS]));
    } else {
        static_assert(MULT == MULT_MHD3, "mult");
        // z+_j = x[j XS], z-_i = x[(3 + i) XS]; T_ij = z-_i z+_j, traceless part
        const X p0 = x[0], p1 = x[XS], p2 = x[2 * XS], m0 = x[3 * XS], m1 = x[4 * XS], m2 = x[5 * XS];
        const X t22 = xmul(m2, p2);
        y[0] = xmul(m0, p1);
        y[YS] = xmul(m0, p2);
        y[2 * YS] = xmul(m1, p0);
        y[3 * YS] = xmul(m1, p2);
        y[4 * YS] = xmul(m2, p0);
        y[5 * YS] = xmul(m2, p1);
        y[6 * YS] = xsub(xmul(m0, p0), t22);
        y[7 * YS] = xsub(xmul(m1, p1), t22);
    }
}

// output b of mult at one point (the OUT_SMEM path, one output at a time)
template <int MULT, int XS, class X>
__device__ __forceinline__ X mult_out(const X* x, int b) {
    static_assert(MULT == MULT_BASD3 || MULT == MULT_MHD3, "outputs one at a time: the 3D Basdevant and MHD mults");
    if constexpr (MULT == MULT_BASD3) {
        const X x0 = x[0], x1 = x[XS], x2 = x[2 * XS];
        switch (b) {
            case 0: return xmul(x0, x1);
            case 1: return xmul(x1, x2);
            case 2: return xmul(x2, x0);
            case 3: return xmul(xadd(x0, x2), xsub(x0, x2));
            default: return xmul(xadd(x1, x2), xsub(x1, x2));
        }
    } else {
        // z+_j = x[j XS], z-_i = x[(3 + i) XS]; T_ij = z-_i z+_j
        const X p0 = x[0], p1 = x[XS], p2 = x[2 * XS], m0 = x[3 * XS], m1 = x[4 * XS], m2 = x[5 * XS];
        switch (b) {
            case 0: return xmul(m0, p1);
            case 1: return xmul(m0, p2);
            case 2: return xmul(m1, p0);
            case 3: return xmul(m1, p2);
            case 4: return xmul(m2, p0);
            case 5: return xmul(m2, p1);
            case 6: return xsub(xmul(m0, p0), xmul(m2, p2));
            default: return xsub(xmul(m1, p1), xmul(m2, p2));
        }
    }
}

struct ConvArgs {
    const void* f[kMaxIn];   // A input bases (device)
    void* h[kMaxOut];   // B output bases (device)
    int64_t stride;     // elements between instances
    int64_t count;      // instances
    int L;              // stored length of complex/centered data; full length for Hermitian
    int Ls;             // stored length (Hermitian: ceil(L/2))
    int H;              // centered offset floor(L/2)
    int n;              // residues
    int N;              // n * S = q * m
    int ls_pad;         // staged row length in shared memory (>= Ls, even)
    const void* twS;    // FFT pass twiddles (FftShape<S, E> layout)
    const void* twN;    // residue twists: zeta_N^{r j} at r S + j (r < n, j < S), then zeta_N^{r S} at n S + r
    double invN;        // 1 / N
    int* err;           // persistent kernel: set to 1 when a bounded wait runs out (may be null)
    int r_begin, r_end; // residues summed: r_begin <= r < r_end (0, n for the whole convolution);
                        // Hermitian pairs start at r_begin
};

template <bool B>
struct BoolTag {
    static constexpr bool value = B;
};

// Conjugate symmetry of the twists (Section 6.3).  Residues r and n - r have
// conjugate twists up to a factor zeta_S^{j}: zeta_N^{(n-r) j} = zeta_S^{j}
// conj(zeta_N^{r j}), since N = n S.  So residue r > n/2 reads the twist row of
// residue n - r and conjugates it; its transform input is then the true one
// times zeta_S^{-j}, whose FFT is the true spectrum shifted by one frequency
// (F'_k = F_{k-1}).  All A inputs shift alike, so the pointwise mult gives the
// shifted product, and the backward transform with the same conjugated twist
// (the conjugate of zeta_S^{-j} conj(zeta_N^{r' j})) puts the contribution back
// in place: zeta_N^{-r' i} IFFT(P)_i = zeta_N^{(n-r') i} IFFT(P')_i.  Residue
// n/2 (even n) pairs with itself and keeps its own row.  Half of the n twist
// rows are read; the block-1 factor zeta_N^{r S} is unchanged.
struct TwistRow {
    int row;     // residue whose table row is read
    bool conj;   // conjugate the entries
};
__host__ __device__ __forceinline__ TwistRow twist_row(int r, int n) {
    return 2 * r > n ? TwistRow{n - r, true} : TwistRow{r, false};
}
template <class T>
__device__ __forceinline__ T twist_ld(const T* p, bool conj) {
    const T w = ldtw(p);
    return conj ? cconj(w) : w;
}

// Residue-sum accumulation.  COMP: TwoSum compensated s + c += x (FP32 path);
// otherwise a plain sum.
template <class R, bool COMP>
__device__ __forceinline__ void acc_add(R& s, R& c, R x) {
    if constexpr (COMP) {
        R t = s + x;
        R bp = t - s;
        R err = (s - (t - bp)) + (x - bp);
        s = t;
        c += err;
    } else {
        s += x;
    }
}

// Input element i: a plain load, or (STREAM) a streaming global load marked
// evict-first, for inputs read once from HBM that should not displace
// L2-resident work buffers.
template <bool STREAM, class T>
__device__ __forceinline__ T ld_in(const T* f, int i) {
    if constexpr (STREAM) return __ldcs(f + i);
    else return f[i];
}
template <bool STREAM, class T>
__device__ __forceinline__ T ld_in(const T* f, int64_t i) {
    if constexpr (STREAM) return __ldcs(f + i);
    else return f[i];
}

// Stored input value(s) folded to transform slot j (see header comment).
// Returns block-0 and block-1 values (block 1 is conj-mirrored for Hermitian).
template <int KIND, bool STREAM = false, class T>
__device__ __forceinline__ void load_fold(const T* f, int j, int S, const ConvArgs& a, bool valid, T& b0, T& b1) {
    b0 = czero<T>();
    b1 = czero<T>();
    if (!valid) return;
    if constexpr (KIND == KIND_COMPLEX) {
        if (j < a.L) b0 = ld_in<STREAM>(f, j);
        if (j + S < a.L) b1 = ld_in<STREAM>(f, j + S);
    } else if constexpr (KIND == KIND_CENTERED) {
        if (j < a.L - a.H) b0 = ld_in<STREAM>(f, j + a.H);
        if (j >= S - a.H) b1 = ld_in<STREAM>(f, j - S + a.H);
    } else {
        if (j < a.Ls) {
            b0 = ld_in<STREAM>(f, j);
            if (j == 0) b0.y = 0;
        }
        if (j > 0 && S - j < a.Ls) b1 = cconj(ld_in<STREAM>(f, S - j));
    }
}

// Block size bound: one group of T threads, or up to 256 threads of groups.
template <int S, int E>
struct ConvLaunch {
    static constexpr int T = S / E;
    static constexpr int MAXT = T > 256 ? T : 256;
};

// Body of one fused convolution for one thread group: instance `inst` of a,
// thread tau of the group, the group's staging area st (A * ls_pad values)
// and exchange buffers sm (A * SMEM values).  Every thread of the CTA runs the
// same sequence of barriers (groups of one CTA share n).  sm holds NX = max(A, B)
// exchange buffers of SMEM values.  FFT twiddles are
// read through the read-only data cache (a shared-memory table measured
// slower: it competes with the exchanges for shared-memory bandwidth).
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// STAGE = false: the inputs are already in st (staged by bulk copies).
// consumed(): called by every thread once the staged inputs are no longer
// read (after the forward transforms of the last residue, whose exchanges
// put barriers after the last reads of st).
template <class R, int S, int E, int KIND, int MULT, int NB, bool COMP, bool STAGE = true, class Hook = NoHook>
__device__ __forceinline__ void conv1d_body(const ConvArgs& a, int64_t inst, bool valid, int tau, cplx<R>* st,
                                            cplx<R>* sm, const Hook& consumed = Hook{}) {
    using T = cplx<R>;
    using Sh = FftShape<S, E>;
    constexpr int TT = Sh::T;
    constexpr int A = MultShape<MULT>::A;
    constexpr int B = MultShape<MULT>::B;
    constexpr bool OSM = MultShape<MULT>::OUT_SMEM;
    constexpr int BR = OSM ? 1 : B;   // outputs whose residue sums live in registers
    const T* twN = static_cast<const T*>(a.twN);
    // pass twiddles: radix-8/16 passes read three or four powers and form the rest
    const TwGlobalProducts<T> twS{static_cast<const T*>(a.twS)};
    // OUT_SMEM: residue sums of output b, block nb at acc[(b NB + nb) S + j], each
    // entry read and written only by the thread that owns slot j
    T* acc = sm + MultShape<MULT>::NX * Sh::SMEM;
    if constexpr (OSM) {
#pragma unroll 1
        for (int b = 0; b < B * NB; ++b)
#pragma unroll
            for (int e = 0; e < E; ++e) acc[b * S + tau + TT * e] = czero<T>();
    }

    if constexpr (STAGE) {
        // stage the A inputs of this convolution in shared memory (coalesced)
        if (valid) {
#pragma unroll
            for (int aa = 0; aa < A; ++aa) {
                const T* src = static_cast<const T*>(a.f[aa]) + inst * a.stride;
                T* dst = st + aa * a.ls_pad;
                for (int i = tau; i < a.Ls; i += TT) dst[i] = __ldcs(src + i);   // streamed: keep L1 for the tables
            }
        }
        __syncthreads();
    }

    // residue sums of output b at [b * 2E + 2e (+1)]
    R s0[BR * 2 * E], c0[COMP ? BR * 2 * E : 1];
    R s1[NB == 2 ? BR * 2 * E : 1], c1[(NB == 2 && COMP) ? BR * 2 * E : 1];
#pragma unroll
    for (int e = 0; e < BR * 2 * E; ++e) s0[e] = R(0);
    if constexpr (COMP) {
#pragma unroll
        for (int e = 0; e < BR * 2 * E; ++e) c0[e] = R(0);
    }
    if constexpr (NB == 2) {
#pragma unroll
        for (int e = 0; e < BR * 2 * E; ++e) s1[e] = R(0);
        if constexpr (COMP) {
#pragma unroll
            for (int e = 0; e < BR * 2 * E; ++e) c1[e] = R(0);
        }
    }
    R dummy = R(0);

    if constexpr (KIND != KIND_HERMITIAN) {
        // residue r; R0: r = 0, whose twists are all 1 (no loads, no multiplies)
        auto residue = [&](int r, auto r0_tag) {
            constexpr bool R0 = decltype(r0_tag)::value;
            const TwistRow tr = twist_row(r, a.n);
            const T* twr = twN + (int64_t)tr.row * S;   // zeta_N^{r j}, j < S (or the paired row, conjugated)
            T cr = R0 ? mk<T>(1, 0) : ldtw(twN + (int64_t)a.n * S + r);    // zeta_N^{r S}
            if constexpr (KIND == KIND_CENTERED) cr = cconj(cr);
            T v[A * E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int j = tau + TT * e;
                const T tw = R0 ? mk<T>(1, 0) : twist_ld(twr + j, tr.conj);
#pragma unroll
                for (int aa = 0; aa < A; ++aa) {
                    if constexpr (KIND == KIND_COMPLEX && NB == 1) {
                        // L <= S: one block, nothing folds in
                        const T* sa = st + aa * a.ls_pad;
                        const T x = (valid && j < a.L) ? sa[j] : czero<T>();
                        v[aa * E + e] = R0 ? x : cmul(x, tw);
                    } else {
                        T b0, b1;
                        load_fold<KIND>(st + aa * a.ls_pad, j, S, a, valid, b0, b1);
                        v[aa * E + e] = R0 ? cadd(b0, b1) : cmul(cadd(b0, cmul(cr, b1)), tw);
                    }
                }
            }
            fft_forward<S, E, A>(v, sm, twS, tau);
            if (r == a.r_end - 1) consumed();
            if constexpr (OSM) {
                T twe[E];
#pragma unroll
                for (int e = 0; e < E; ++e) twe[e] = R0 ? mk<T>(1, 0) : twist_ld(twr + tau + TT * e, tr.conj);
#pragma unroll 1
                for (int b = 0; b < B; ++b) {
                    T p[E];
#pragma unroll
                    for (int e = 0; e < E; ++e) p[e] = mult_out<MULT, E>(v + e, b);
                    fft_inverse<S, E, 1>(p, sm, twS, tau);
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int j = tau + TT * e;
                        const T y = R0 ? p[e] : cmulc(p[e], twe[e]);      // zeta_N^{-r j} y_j
                        T* q0 = acc + (b * NB) * S + j;
                        *q0 = cadd(*q0, y);
                        if constexpr (NB == 2) {
                            T* q1 = acc + (b * NB + 1) * S + j;
                            *q1 = cadd(*q1, R0 ? y : cmulc(y, cr));     // block 1: extra zeta_N^{-r S}
                        }
                    }
                }
                return;
            }
            T p[B * E];
#pragma unroll
            for (int e = 0; e < E; ++e) mult_point<MULT, E, E>(v + e, p + e);
            fft_inverse<S, E, B>(p, sm, twS, tau);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int j = tau + TT * e;
                const T tw = R0 ? mk<T>(1, 0) : twist_ld(twr + j, tr.conj);
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    const int o = b * 2 * E + 2 * e;
                    const T y = R0 ? p[b * E + e] : cmulc(p[b * E + e], tw);   // zeta_N^{-r j} y_j
                    acc_add<R, COMP>(s0[o], COMP ? c0[o] : dummy, y.x);
                    acc_add<R, COMP>(s0[o + 1], COMP ? c0[o + 1] : dummy, y.y);
                    if constexpr (NB == 2) {
                        const T y1 = R0 ? y : cmulc(y, cr);             // block 1: extra zeta_N^{-r o}
                        acc_add<R, COMP>(s1[o], COMP ? c1[o] : dummy, y1.x);
                        acc_add<R, COMP>(s1[o + 1], COMP ? c1[o + 1] : dummy, y1.y);
                    }
                }
            }
        };
        if (a.r_begin == 0) residue(0, BoolTag<true>{});
        for (int r = a.r_begin > 0 ? a.r_begin : 1; r < a.r_end; ++r) residue(r, BoolTag<false>{});
    } else {
        // residue pair (r1, r1 + 1); R0: r1 = 0, whose twists are all 1
        auto pair = [&](int r1, auto r0_tag) {
            constexpr bool R0 = decltype(r0_tag)::value;
            const int r2 = r1 + 1;
            const bool has2 = r2 < a.r_end;
            const T* twr1 = twN + (int64_t)r1 * S;
            const T* twr2 = twN + (int64_t)(has2 ? r2 : r1) * S;
            const T cr1 = R0 ? mk<T>(1, 0) : cconj(ldtw(twN + (int64_t)a.n * S + r1));      // zeta_N^{-r1 S}
            const T cr2 = has2 ? cconj(ldtw(twN + (int64_t)a.n * S + r2)) : czero<T>();
            T v[A * E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int j = tau + TT * e;
                const T t1 = R0 ? mk<T>(1, 0) : ldtw(twr1 + j);
                const T t2 = has2 ? ldtw(twr2 + j) : czero<T>();
#pragma unroll
                for (int aa = 0; aa < A; ++aa) {
                    T b0, b1;
                    load_fold<KIND>(st + aa * a.ls_pad, j, S, a, valid, b0, b1);
                    const T w1 = R0 ? cadd(b0, b1) : cmul(cadd(b0, cmul(cr1, b1)), t1);
                    const T w2 = cmul(cadd(b0, cmul(cr2, b1)), t2);
                    v[aa * E + e] = mk<T>(w1.x - w2.y, w1.y + w2.x);   // W1 + i W2
                }
            }
            fft_forward<S, E, A>(v, sm, twS, tau);
            if (r1 + 2 >= a.r_end) consumed();
            if constexpr (OSM) {
#pragma unroll 1
                for (int b = 0; b < B; ++b) {
                    T p[E];
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        R xr[A], xi[A];
#pragma unroll
                        for (int aa = 0; aa < A; ++aa) {
                            xr[aa] = v[aa * E + e].x;
                            xi[aa] = v[aa * E + e].y;
                        }
                        p[e] = mk<T>(mult_out<MULT, 1>(xr, b), mult_out<MULT, 1>(xi, b));
                    }
                    fft_inverse<S, E, 1>(p, sm, twS, tau);
#pragma unroll
                    for (int e = 0; e < E; ++e) sm[padidx(tau + TT * e)] = p[e];
                    __syncthreads();
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int j = tau + TT * e;
                        const T t1 = R0 ? mk<T>(1, 0) : ldtw(twr1 + j);
                        const T t2 = has2 ? ldtw(twr2 + j) : czero<T>();
                        const T ym = sm[padidx((S - j) & (S - 1))];
                        const T yj = p[e];
                        const R hf = R(0.5);
                        const T g1 = mk<T>((yj.x + ym.x) * hf, (yj.y - ym.y) * hf);
                        const T d = mk<T>(yj.x - ym.x, yj.y + ym.y);
                        const T g2 = mk<T>(d.y * hf, -d.x * hf);
                        T y = R0 ? g1 : cmulc(g1, t1);
                        if (has2) y = cadd(y, cmulc(g2, t2));
                        T* q = acc + b * S + j;
                        *q = cadd(*q, y);
                    }
                    __syncthreads();
                }
                return;
            }
            // real parts carry residue r1, imaginary parts residue r2: mult on each
            T p[B * E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                R xr[A], xi[A], yr[B], yi[B];
#pragma unroll
                for (int aa = 0; aa < A; ++aa) {
                    xr[aa] = v[aa * E + e].x;
                    xi[aa] = v[aa * E + e].y;
                }
                mult_point<MULT, 1, 1>(xr, yr);
                mult_point<MULT, 1, 1>(xi, yi);
#pragma unroll
                for (int b = 0; b < B; ++b) p[b * E + e] = mk<T>(yr[b], yi[b]);
            }
            fft_inverse<S, E, B>(p, sm, twS, tau);
            // split the two Hermitian inverses: needs Y_{S-j} (output b in exchange buffer b)
#pragma unroll
            for (int e = 0; e < E; ++e) {
#pragma unroll
                for (int b = 0; b < B; ++b) sm[b * Sh::SMEM + padidx(tau + TT * e)] = p[b * E + e];
            }
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int j = tau + TT * e;
                const T t1 = R0 ? mk<T>(1, 0) : ldtw(twr1 + j);
                const T t2 = has2 ? ldtw(twr2 + j) : czero<T>();
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    const int o = b * 2 * E + 2 * e;
                    const T ym = sm[b * Sh::SMEM + padidx((S - j) & (S - 1))];
                    const T yj = p[b * E + e];
                    const R hf = R(0.5);
                    const T g1 = mk<T>((yj.x + ym.x) * hf, (yj.y - ym.y) * hf);   // (Y_j + conj Y_{S-j}) / 2
                    const T d = mk<T>(yj.x - ym.x, yj.y + ym.y);                  // Y_j - conj Y_{S-j}
                    const T g2 = mk<T>(d.y * hf, -d.x * hf);                       // d / (2i)
                    T y = R0 ? g1 : cmulc(g1, t1);
                    if (has2) y = cadd(y, cmulc(g2, t2));
                    acc_add<R, COMP>(s0[o], COMP ? c0[o] : dummy, y.x);
                    acc_add<R, COMP>(s0[o + 1], COMP ? c0[o + 1] : dummy, y.y);
                }
            }
            __syncthreads();
        };
        if (a.r_begin == 0) pair(0, BoolTag<true>{});
        for (int r1 = a.r_begin > 0 ? a.r_begin : 2; r1 < a.r_end; r1 += 2) pair(r1, BoolTag<false>{});
    }

    if (!valid) return;
    const R sc = R(a.invN);
#pragma unroll
    for (int b = 0; b < B; ++b) {
        T* hout = static_cast<T*>(a.h[b]) + inst * a.stride;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int j = tau + TT * e;
            T o0, o1 = czero<T>();
            if constexpr (OSM) {
                o0 = cscale(acc[(b * NB) * S + j], sc);
                if constexpr (NB == 2) o1 = cscale(acc[(b * NB + 1) * S + j], sc);
            } else {
                const int o = b * 2 * E + 2 * e;
                const R x0 = COMP ? s0[o] + c0[o] : s0[o];
                const R y0 = COMP ? s0[o + 1] + c0[o + 1] : s0[o + 1];
                o0 = mk<T>(x0 * sc, y0 * sc);
                if constexpr (NB == 2) {
                    const R x1 = COMP ? s1[o] + c1[o] : s1[o];
                    const R y1 = COMP ? s1[o + 1] + c1[o + 1] : s1[o + 1];
                    o1 = mk<T>(x1 * sc, y1 * sc);
                }
            }
            if constexpr (KIND == KIND_COMPLEX) {
                if (j < a.L) __stcs(hout + j, o0);
                if constexpr (NB == 2) {
                    if (j + S < a.L) __stcs(hout + j + S, o1);
                }
            } else if constexpr (KIND == KIND_CENTERED) {
                if (j < a.L - a.H) __stcs(hout + j + a.H, o0);
                if constexpr (NB == 2) {
                    if (j >= S - a.H) __stcs(hout + j - S + a.H, o1);
                }
            } else {
                if (j < a.Ls) __stcs(hout + j, o0);
            }
        }
    }
}

// One thread group of T = S/E threads per convolution; G = blockDim.x / T
// groups per CTA; shared memory per group: the A staged inputs (ls_pad values
// each), then A padded FFT exchange buffers.  MINB: CTAs per SM the register
// allocation must allow (1: up to 255 registers for 256 threads; 2: at most
// 128; the MINB = 2 variants up to S = 256 are held to three CTAs per SM, 80
// registers: their rows are short, and the third CTA hides more of the staging
// loads, 2 % on the 256^3 Hermitian plan, whose inner rows are S = 128).
template <class R, int S, int E, int KIND, int MULT, int NB, bool COMP, int MINB>
__global__ void __launch_bounds__(ConvLaunch<S, E>::MAXT, (MINB == 2 && S <= 256) ? 3 : MINB)
    conv1d_kernel(const __grid_constant__ ConvArgs a) {
    using T = cplx<R>;
    using Sh = FftShape<S, E>;
    constexpr int TT = Sh::T;
    constexpr int A = MultShape<MULT>::A;
    constexpr int NX = MultShape<MULT>::NX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = blockDim.x / TT;
    const int g = threadIdx.x / TT;
    const int tau = threadIdx.x - g * TT;
    T* st = reinterpret_cast<T*>(smem_raw) + (size_t)g * (A * a.ls_pad + NX * Sh::SMEM + MultShape<MULT>::acc(S));
    T* sm = st + A * a.ls_pad;
    const int64_t inst = (int64_t)blockIdx.x * G + g;
    conv1d_body<R, S, E, KIND, MULT, NB, COMP>(a, inst, inst < a.count, tau, st, sm);
}

// ---------------------------------------------------------------------------
// Persistent variant with double-buffered staging by bulk copies.
//
// One CTA per SM loops over its share of the batch.  Thread 0 stages the
// inputs of the next convolution(s) into the second staging buffer with
// cp.async.bulk (the TMA engine copies global -> shared, completion counted
// on an mbarrier) while the CTA computes on the first, so the HBM latency of
// the next batch element is hidden behind the current one's transforms.
// Rows must start on 16-byte boundaries and span a multiple of 16 bytes
// (checked by the launcher).  Every wait on an mbarrier is bounded in time:
// a wait that runs out sets *err to 1 and the CTA returns after a bounded
// wait for its other copy in flight.

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// thread 0: expect `bytes` of transactions on bar and arrive
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ long long conv_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

// bounded wait for the phase with the given parity (about 2 s)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const long long t0 = conv_ns();
    while (!mbar_try(bar, parity))
        if (conv_ns() - t0 > 2000000000LL) return false;
    return true;
}

// NBUF = 1 (the launchers' choice): one buffer, released early: the copy for
// the next step starts once the last residue's forward transforms have
// consumed the staged inputs, and overlaps that residue's product, inverse
// transform and accumulation.  NBUF = 2: the next step is staged into a second
// buffer while the CTA computes.
template <class R, int S, int E, int KIND, int MULT, int NB, bool COMP, int MINB, int NBUF>
__global__ void __launch_bounds__(ConvLaunch<S, E>::MAXT, MINB) conv1d_kernel_pipe(const __grid_constant__ ConvArgs a) {
    using T = cplx<R>;
    using Sh = FftShape<S, E>;
    constexpr int TT = Sh::T;
    constexpr int A = MultShape<MULT>::A;
    constexpr int NX = MultShape<MULT>::NX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_ok;
    const int G = blockDim.x / TT;
    const int g = threadIdx.x / TT;
    const int tau = threadIdx.x - g * TT;
    const size_t stage_elems = (size_t)G * A * a.ls_pad;          // one staging buffer (all groups)
    T* stage0 = reinterpret_cast<T*>(smem_raw);
    T* sm = stage0 + NBUF * stage_elems + (size_t)g * (NX * Sh::SMEM + MultShape<MULT>::acc(S));
    const int64_t nsteps = (a.count + G - 1) / G;                    // CTA steps over the batch
    const uint32_t row_bytes = (uint32_t)(a.Ls * sizeof(T));

    // thread 0: stage step `k` (G convolutions) into buffer b
    auto issue = [&](int64_t k, int b) {
        uint32_t bytes = 0;
        for (int gg = 0; gg < G; ++gg)
            if (k * G + gg < a.count) bytes += A * row_bytes;
        mbar_expect(&bar[b], bytes);
        for (int gg = 0; gg < G; ++gg) {
            const int64_t inst = k * G + gg;
            if (inst >= a.count) break;
#pragma unroll
            for (int aa = 0; aa < A; ++aa)
                bulk_g2s(stage0 + b * stage_elems + ((size_t)gg * A + aa) * a.ls_pad,
                         static_cast<const T*>(a.f[aa]) + inst * a.stride, row_bytes, &bar[b]);
        }
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    int64_t k = blockIdx.x;
    if (k >= nsteps) return;
    if (threadIdx.x == 0) issue(k, 0);
    for (int it = 0; k < nsteps; ++it, k += gridDim.x) {
        const int b = NBUF == 2 ? (it & 1) : 0;
        const uint32_t parity = NBUF == 2 ? (uint32_t)((it >> 1) & 1) : (uint32_t)(it & 1);
        const int64_t kn = k + gridDim.x;
        if (NBUF == 2 && threadIdx.x == 0 && kn < nsteps) issue(kn, b ^ 1);   // released by the last barrier
        if (threadIdx.x == 0) s_ok = mbar_wait(&bar[b], parity) ? 1 : 0;
        __syncthreads();
        if (!s_ok) {
            if (threadIdx.x == 0) {
                // the copies this CTA issued may still be in flight: wait for each once
                // more (bounded) before the CTA leaves; 2 records that one had not landed
                int code = 1;
                if (!mbar_wait(&bar[b], parity)) code = 2;
                if (NBUF == 2 && kn < nsteps && !mbar_wait(&bar[b ^ 1], (uint32_t)(((it + 1) >> 1) & 1))) code = 2;
                if (a.err) atomicMax(a.err, code);
            }
            return;
        }
        mbar_try(&bar[b], parity);                                   // this thread's own acquire of the phase
        const int64_t inst = k * G + g;
        T* st = stage0 + b * stage_elems + (size_t)g * A * a.ls_pad;
        if constexpr (NBUF == 2) {
            conv1d_body<R, S, E, KIND, MULT, NB, COMP, false>(a, inst, inst < a.count, tau, st, sm);
        } else {
            auto release = [&]() {
                __syncthreads();                                     // every thread is past its last read of st
                if (threadIdx.x == 0 && kn < nsteps) issue(kn, 0);
            };
            conv1d_body<R, S, E, KIND, MULT, NB, COMP, false>(a, inst, inst < a.count, tau, st, sm, release);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Cluster variant for few convolutions (D > 1 residues per pass, Section 6.5).
//
// A convolution that runs alone on one CTA is bound by that SM's arithmetic
// (most of all in FP64).  Residue contributions are independent and add up
// (Section 2.2), so here one convolution runs on a thread-block cluster of
// D * A CTAs: CTA c takes residue group g = c / A (residues r = g, g + D, ...)
// and input ai = c % A.  Per residue, every CTA folds, twists and transforms
// its own input; the CTAs with ai > 0 publish their spectra in shared memory
// (two buffers, alternating between residues); after a cluster barrier the
// group's CTA ai = 0 reads them through distributed shared memory, applies
// mult, runs the inverse transform and accumulates.  At the end each group's
// scaled partial sums are written to shared memory, and every CTA of the
// cluster sums a slice of the outputs over the D groups in a fixed order
// (deterministic) and stores it.  Complex and centered kinds, one output.
// Residue sums are plain.  A lone convolution is latency-bound, so each CTA
// copies its FFT twiddles into shared memory once, together with the input
// row, and each residue's twist row before its fold.
template <class R, int S, int E, int KIND, int MULT, int NB>
__global__ void __launch_bounds__(S / E) conv1d_cluster_kernel(const __grid_constant__ ConvArgs a, int D) {
    using T = cplx<R>;
    using Sh = FftShape<S, E>;
    constexpr int TT = Sh::T;
    constexpr int A = MultShape<MULT>::A;
    static_assert(MultShape<MULT>::B == 1 && KIND != KIND_HERMITIAN, "cluster variant: one output, not Hermitian");
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int CL = D * A;
    const int c = (int)cl.block_rank();
    const int g = c / A, ai = c - g * A;
    const int64_t inst = blockIdx.x / CL;
    const int tau = threadIdx.x;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* st = reinterpret_cast<T*>(smem_raw);   // staged input ai (ls_pad values); the partial sums at the end
    T* sm = st + a.ls_pad;                      // FFT exchange buffer
    T* spec = sm + Sh::SMEM;                    // published spectra: two buffers of S values
    T* tws = spec + 2 * S;                      // FFT pass twiddles (TW_TOTAL values)
    T* twr = tws + (Sh::TW_TOTAL > 0 ? Sh::TW_TOTAL : 1);   // twists of the current residue (S values)
    const T* twN = static_cast<const T*>(a.twN);
    const T* twg = static_cast<const T*>(a.twS);
    const TwShared<T> twS{tws};
    const T* src = static_cast<const T*>(a.f[ai]) + inst * a.stride;
    for (int i = tau; i < a.Ls; i += TT) st[i] = src[i];
    for (int i = tau; i < Sh::TW_TOTAL; i += TT) tws[i] = __ldg(twg + i);
    __syncthreads();

    R s0[2 * E], s1[NB == 2 ? 2 * E : 1];
#pragma unroll
    for (int e = 0; e < 2 * E; ++e) {
        s0[e] = R(0);
        if constexpr (NB == 2) s1[e] = R(0);
    }
    R dummy = R(0);
    const int nsteps = (a.r_end - a.r_begin + D - 1) / D;
    for (int k = 0; k < nsteps; ++k) {
        const int r = a.r_begin + g + k * D;
        const bool act = r < a.r_end;         // uniform over the CTA
        T* spk = spec + (k & 1) * S;
        T cr = ldtw(twN + (int64_t)a.n * S + (act ? r : 0));   // zeta_N^{r S}
        if constexpr (KIND == KIND_CENTERED) cr = cconj(cr);
        T v[E];
        if (act) {
            // this residue's twists zeta_N^{r j}, once every thread has finished
            // the previous residue's accumulation (which reads the old row)
            __syncthreads();
            const TwistRow tr = twist_row(r, a.n);   // conjugate symmetry (see twist_row)
            const T* row = twN + (int64_t)tr.row * S;
            for (int i = tau; i < S; i += TT) twr[i] = twist_ld(row + i, tr.conj);
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int j = tau + TT * e;
                const T tw = twr[j];
                if constexpr (KIND == KIND_COMPLEX && NB == 1) {
                    const T x = j < a.L ? st[j] : czero<T>();
                    v[e] = cmul(x, tw);
                } else {
                    T b0, b1;
                    load_fold<KIND>(st, j, S, a, true, b0, b1);
                    v[e] = cmul(cadd(b0, cmul(cr, b1)), tw);
                }
            }
            fft_forward<S, E, 1>(v, sm, twS, tau);
            if (ai != 0) {
#pragma unroll
                for (int e = 0; e < E; ++e) spk[e * TT + tau] = v[e];
            }
        }
        cl.sync();                             // spectra of residue r published
        if (act && ai == 0) {
            T x[A * E];
#pragma unroll
            for (int e = 0; e < E; ++e) x[e] = v[e];
#pragma unroll
            for (int aa = 1; aa < A; ++aa) {
                const T* rem = cl.map_shared_rank(spk, (unsigned)(g * A + aa));
#pragma unroll
                for (int e = 0; e < E; ++e) x[aa * E + e] = rem[e * TT + tau];
            }
            T p[E];
#pragma unroll
            for (int e = 0; e < E; ++e) mult_point<MULT, E, E>(x + e, p + e);
            fft_inverse<S, E, 1>(p, sm, twS, tau);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int j = tau + TT * e;
                const T y = cmulc(p[e], twr[j]);          // zeta_N^{-r j} y_j
                acc_add<R, false>(s0[2 * e], dummy, y.x);
                acc_add<R, false>(s0[2 * e + 1], dummy, y.y);
                if constexpr (NB == 2) {
                    const T y1 = cmulc(y, cr);            // block 1: extra zeta_N^{-r S}
                    acc_add<R, false>(s1[2 * e], dummy, y1.x);
                    acc_add<R, false>(s1[2 * e + 1], dummy, y1.y);
                }
            }
        }
        // the next residue publishes into the other buffer; the one after that
        // reuses this one only after the next cluster barrier, which every
        // reader of this buffer reaches after its reads
    }
    __syncthreads();                           // st is no longer read: it takes the partial sums
    if (ai == 0) {
        const R sc = R(a.invN);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int j = tau + TT * e;
            const T o0 = mk<T>(s0[2 * e] * sc, s0[2 * e + 1] * sc);
            if constexpr (KIND == KIND_COMPLEX) {
                if (j < a.L) st[j] = o0;
                if constexpr (NB == 2) {
                    if (j + S < a.L) st[j + S] = mk<T>(s1[2 * e] * sc, s1[2 * e + 1] * sc);
                }
            } else {
                if (j < a.L - a.H) st[j + a.H] = o0;
                if (j >= S - a.H) st[j - S + a.H] = mk<T>(s1[2 * e] * sc, s1[2 * e + 1] * sc);
            }
        }
    }
    cl.sync();                                 // partial sums of every group written
    const int chunk = (a.Ls + CL - 1) / CL;
    const int i1 = (c + 1) * chunk < a.Ls ? (c + 1) * chunk : a.Ls;
    T* hout = static_cast<T*>(a.h[0]) + inst * a.stride;
    for (int i = c * chunk + tau; i < i1; i += TT) {
        T sum = czero<T>();
        for (int gg = 0; gg < D; ++gg) sum = cadd(sum, cl.map_shared_rank(st, (unsigned)(gg * A))[i]);
        hout[i] = sum;
    }
    cl.sync();                                 // no CTA leaves while others read its shared memory
}

// Forward transform of one residue of one input, written in the paper's
// order: out[u m + l] = X[P l + u] with P = S/m (see hd_forward_residue).
template <class R, int S, int E, int KIND>
__global__ void __launch_bounds__(S / E) forward_residue_kernel(const __grid_constant__ ConvArgs a, int r, int m,
                                                               void* out) {
    using T = cplx<R>;
    using Sh = FftShape<S, E>;
    constexpr int TT = Sh::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int tau = threadIdx.x;
    const TwGlobal<T> twS{static_cast<const T*>(a.twS)};
    const T* twN = static_cast<const T*>(a.twN);
    const T* f = static_cast<const T*>(a.f[0]);
    T cr = ldtw(twN + (int64_t)a.n * S + r);
    if constexpr (KIND != KIND_COMPLEX) cr = cconj(cr);
    T v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int j = tau + TT * e;
        T b0, b1;
        load_fold<KIND>(f, j, S, a, true, b0, b1);
        v[e] = cmul(cadd(b0, cmul(cr, b1)), ldtw(twN + (int64_t)r * S + j));
    }
    fft_forward<S, E>(v, sm, twS, tau);
    const int P = S / m;
    T* o = static_cast<T*>(out);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = spectral_index<S, E>(tau, e);
        T x = v[e];
        if constexpr (KIND == KIND_HERMITIAN) x.y = 0;
        o[(k % P) * m + k / P] = x;
    }
}

}  // namespace hd
