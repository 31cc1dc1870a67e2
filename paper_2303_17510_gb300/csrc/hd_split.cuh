// hd_split.cuh -- residue transforms larger than one CTA (the "split" path).
//
// A residue transform of size S = S1 * S2 (S2 <= the fused limit, S1 <= 16)
// is computed in the order of the paper's inner loop (Section 6.1,
// forwardInner / backwardInner): size-S1 DFTs along the block index t (here
// j1), the twiddle zeta_S^{j2 k1}, then size-S2 FFTs along s (here j2):
//     X_{k1 + S1 k2} = sum_{j2} zeta_{S2}^{j2 k2} zeta_S^{j2 k1}
//                      sum_{j1} zeta_{S1}^{j1 k1} W_{j1 S2 + j2}.
// Three kernels per batch chunk, with the work buffer of Section 5 (A n S
// values per instance) in device scratch; inputs are read and outputs written
// with evict-first hints so that the work buffer stays in L2 between phases:
//   split_colfwd : per (instance, input a, residue r, column j2): fold and twist
//                  the stored input into W_{j1 S2 + j2}, DFT over j1, twiddle,
//                  store row k1 of the work buffer;
//   split_row    : per (instance, residue, row k1): FFT_{S2} of the A rows, mult,
//                  inverse FFT_{S2}, result written over row k1 of input 0;
//   split_colbwd : per (instance, column j2): for every residue the conjugate
//                  twiddle and inverse DFT over k1, then the residue contribution
//                  zeta_N^{-r i} y_{i mod S} accumulated into the output (all
//                  residues in registers, one store).
// Residues may run in blocks r0 .. r0 + nr - 1 (D residues per pass, Section
// 6.5): the work buffer then holds A nr S values per instance, and the blocks
// after the first add their contributions to the output (the output is the
// accumulation buffer, so none is needed besides it).
// Hermitian residues are not paired here: the residue's spectrum is real and
// the inverse of a real spectrum is Hermitian, so y is used directly.
#pragma once

#include <type_traits>

#include "hd_conv1d.cuh"

namespace hd {

struct SplitArgs {
    const void* f[kMaxIn];   // A input bases
    void* h[kMaxOut];        // B output bases
    int64_t stride;     // elements between instances
    int64_t count;      // instances in this chunk
    int L, Ls, H;       // as ConvArgs
    int n;              // residues
    int S, S1, S2;      // transform size and its split
    int A, B;           // inputs, outputs
    int P;              // work-buffer parts per instance: max(A, B) (output b is written over part b)
    const void* twS;    // zeta_S^{j2 k1} at k1 S2 + j2 (k1 < S1, j2 < S2)
    const void* twR;    // residue twists (ConvArgs::twN layout)
    const void* twS2;   // FFT pass twiddles of the size-S2 row FFT
    void* work;         // scratch: [instance][part < P][r - r0][k1][j2]
    double invN;
    int r0, nr;         // residue block: residues r0 .. r0 + nr - 1
    int accumulate;     // colbwd: add to the output (blocks after the first)
};

template <int S1, bool INV, class T>
__device__ __forceinline__ void dft_small(T* v) {
    dft_reg<S1, INV>(v);
}

// Drops the L2 lines of a work-buffer region whose values are dead, without
// writing them back to DRAM (the region's contents become undefined until it
// is written again).  The region starts on a 128-byte boundary and spans a
// multiple of 128 bytes; threads tid = 0 .. nthreads-1 share the lines.
__device__ __forceinline__ void l2_discard(const void* p, int64_t bytes, int tid, int nthreads) {
    const char* c = static_cast<const char*>(p);
    for (int64_t off = (int64_t)tid * 128; off < bytes; off += (int64_t)nthreads * 128)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(c + off) : "memory");
}

// Twist zeta_N^{r j}, j = j1 S2 + j2, of residue row twr (= twR + r S): the
// product of tb = zeta_N^{r j2} (one read per column) and the row's entry
// j1 S2 = zeta_N^{r j1 S2}, the same for every column (a broadcast read), so a
// column reads S1 + 1 twist entries of which S1 are shared, instead of S1 of
// its own from a table of n S entries.
// With conjugate symmetry (twist_row) both factors come from the paired row,
// conjugated: tb is loaded conjugated, the shared factor here.
template <class T>
__device__ __forceinline__ T split_twist(const T* twr, T tb, int j1, int S2, bool conj) {
    return j1 == 0 ? tb : cmul(tb, twist_ld(twr + (int64_t)j1 * S2, conj));
}

// Forward column j2 of residue r of input aa of instance inst.
template <class R, int S1, int KIND>
__device__ __forceinline__ void split_colfwd_body(const SplitArgs& a, int64_t inst, int aa, int r, int j2) {
    using T = cplx<R>;
    const T* f = static_cast<const T*>(a.f[aa]) + inst * a.stride;
    const T* twR = static_cast<const T*>(a.twR);
    const T* twS = static_cast<const T*>(a.twS);
    ConvArgs ca;
    ca.L = a.L;
    ca.Ls = a.Ls;
    ca.H = a.H;
    T cr = ldtw(twR + (int64_t)a.n * a.S + r);      // zeta_N^{r S}
    if constexpr (KIND != KIND_COMPLEX) cr = cconj(cr);
    const TwistRow tr = twist_row(r, a.n);            // conjugate symmetry
    const T* twr = twR + (int64_t)tr.row * a.S;
    const T tb = twist_ld(twr + j2, tr.conj);         // zeta_N^{r j2}
    T v[S1];
#pragma unroll
    for (int j1 = 0; j1 < S1; ++j1) {
        const int j = j1 * a.S2 + j2;
        T b0, b1;
        load_fold<KIND, true>(f, j, a.S, ca, true, b0, b1);
        v[j1] = cmul(cadd(b0, cmul(cr, b1)), split_twist(twr, tb, j1, a.S2, tr.conj));
    }
    dft_small<S1, false>(v);
    T tw[S1];
    power_row_twiddles<S1, true>(twS + j2, a.S2, tw);   // zeta_S^{j2 k1}
    T* w = static_cast<T*>(a.work) + ((inst * a.P + aa) * a.nr + (r - a.r0)) * (int64_t)a.S;
#pragma unroll
    for (int k1 = 0; k1 < S1; ++k1) {
        const T t = k1 == 0 ? v[0] : cmul(v[k1], tw[k1]);
        w[(int64_t)k1 * a.S2 + j2] = t;
    }
}

// U columns j2 = j2base + u * jstep of one (instance, input, residue) by one
// thread: every load of the U columns is issued before the first store, so a
// thread keeps U * S1 loads in flight (the persistent ragged kernel runs one
// CTA per SM and relies on this for latency hiding).
template <class R, int S1, int KIND, int U>
__device__ __forceinline__ void split_colfwd_multi(const SplitArgs& a, int64_t inst, int aa, int r, int j2base,
                                                   int jstep) {
    using T = cplx<R>;
    const T* f = static_cast<const T*>(a.f[aa]) + inst * a.stride;
    const T* twR = static_cast<const T*>(a.twR);
    const T* twS = static_cast<const T*>(a.twS);
    ConvArgs ca;
    ca.L = a.L;
    ca.Ls = a.Ls;
    ca.H = a.H;
    T cr = ldtw(twR + (int64_t)a.n * a.S + r);      // zeta_N^{r S}
    if constexpr (KIND != KIND_COMPLEX) cr = cconj(cr);
    const TwistRow tr = twist_row(r, a.n);            // conjugate symmetry
    const T* twr = twR + (int64_t)tr.row * a.S;
    T v[U][S1];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int j2 = j2base + u * jstep;
        const T tb = twist_ld(twr + j2, tr.conj);     // zeta_N^{r j2}
#pragma unroll
        for (int j1 = 0; j1 < S1; ++j1) {
            const int j = j1 * a.S2 + j2;
            T b0, b1;
            load_fold<KIND, true>(f, j, a.S, ca, true, b0, b1);
            v[u][j1] = cmul(cadd(b0, cmul(cr, b1)), split_twist(twr, tb, j1, a.S2, tr.conj));
        }
    }
    T* w = static_cast<T*>(a.work) + ((inst * a.P + aa) * a.nr + (r - a.r0)) * (int64_t)a.S;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int j2 = j2base + u * jstep;
        dft_small<S1, false>(v[u]);
        T tw[S1];
        power_row_twiddles<S1, true>(twS + j2, a.S2, tw);   // zeta_S^{j2 k1}
#pragma unroll
        for (int k1 = 0; k1 < S1; ++k1) {
            const T t = k1 == 0 ? v[u][0] : cmul(v[u][k1], tw[k1]);
            w[(int64_t)k1 * a.S2 + j2] = t;
        }
    }
}

// Forward columns: one thread per (instance, a, r, j2), j2 fastest.
template <class R, int S1, int KIND>
__global__ void __launch_bounds__(256) split_colfwd(const __grid_constant__ SplitArgs a) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = a.count * a.A * a.nr * (int64_t)a.S2;
    if (tid >= total) return;
    const int j2 = (int)(tid % a.S2);
    int64_t rest = tid / a.S2;
    const int r = a.r0 + (int)(rest % a.nr);
    rest /= a.nr;
    const int aa = (int)(rest % a.A);
    split_colfwd_body<R, S1, KIND>(a, rest / a.A, aa, r, j2);
}

// Row `row` (= (instance * n + r) * S1 + k1) for one group of S2/E threads;
// sm is the group's exchange buffers (NX of MultShape<MULT>).  The A input
// rows are transformed together, mult forms the B output spectra (together for
// B <= 2, one at a time with the residue spectra in registers for more), and
// output b is written over part b of the work buffer.
// DISCARD: drop the dead input rows a >= 1 from L2 once they are loaded (the
// persistent ragged kernel, whose work buffers would otherwise be written back
// to DRAM; measured slower than leaving them for the batched kernels).
template <class R, int S2, int E, int KIND, int MULT, bool DISCARD = false>
__device__ __forceinline__ void split_row_body(const SplitArgs& a, int64_t row, bool valid, int tau, cplx<R>* sm) {
    using T = cplx<R>;
    using Sh = FftShape<S2, E>;
    constexpr int TT = Sh::T;
    constexpr int A = MultShape<MULT>::A;
    constexpr int B = MultShape<MULT>::B;
    static_assert(!DISCARD || B == 1, "dead-row discards assume one output");
    const int k1 = (int)(row % a.S1);
    const int64_t rr = row / a.S1;
    const int rb = (int)(rr % a.nr);   // residue a.r0 + rb
    const int64_t inst = rr / a.nr;
    const TwGlobalProducts<T> tw{static_cast<const T*>(a.twS2)};
    T* base = static_cast<T*>(a.work);
    auto row_of = [&](int part) { return base + ((inst * a.P + part) * a.nr + rb) * (int64_t)a.S + (int64_t)k1 * S2; };
    T v[A * E];
#pragma unroll
    for (int aa = 0; aa < A; ++aa) {
        const T* src = row_of(aa);
#pragma unroll
        for (int e = 0; e < E; ++e) v[aa * E + e] = valid ? src[tau + TT * e] : czero<T>();
    }
    fft_forward<S2, E, A>(v, sm, tw, tau);
    // rows a >= 1 are dead once every thread has loaded them (the forward
    // transform's exchanges put barriers in between); row 0 receives the result
    if (DISCARD && valid) {
#pragma unroll
        for (int aa = 1; aa < A; ++aa) l2_discard(row_of(aa), (int64_t)S2 * sizeof(T), tau, TT);
    }
    // mult at slot e: Hermitian residue spectra are real, so mult acts on the real parts
    auto spec_in = [&](int e, auto* x) {
#pragma unroll
        for (int aa = 0; aa < A; ++aa) {
            if constexpr (KIND == KIND_HERMITIAN) x[aa] = v[aa * E + e].x;
            else x[aa] = v[aa * E + e];
        }
    };
    using X = std::conditional_t<KIND == KIND_HERMITIAN, R, T>;
    auto as_cplx = [](X y) -> T {
        if constexpr (KIND == KIND_HERMITIAN) return mk<T>(y, R(0));
        else return y;
    };
    if constexpr (MultShape<MULT>::OUT_SMEM) {
#pragma unroll 1
        for (int b = 0; b < B; ++b) {
            T p[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                X x[A];
                spec_in(e, x);
                p[e] = as_cplx(mult_out<MULT, 1>(x, b));
            }
            fft_inverse<S2, E, 1>(p, sm, tw, tau);
            if (valid) {
                T* dst = row_of(b);
#pragma unroll
                for (int e = 0; e < E; ++e) dst[tau + TT * e] = p[e];
            }
        }
    } else {
        T p[B * E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            X x[A], y[B];
            spec_in(e, x);
            mult_point<MULT, 1, 1>(x, y);
#pragma unroll
            for (int b = 0; b < B; ++b) p[b * E + e] = as_cplx(y[b]);
        }
        fft_inverse<S2, E, B>(p, sm, tw, tau);
        if (!valid) return;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            T* dst = row_of(b);
#pragma unroll
            for (int e = 0; e < E; ++e) dst[tau + TT * e] = p[b * E + e];
        }
    }
}

// Rows: one group of S2/E threads per (instance, residue, row k1).
template <class R, int S2, int E, int KIND, int MULT>
__global__ void __launch_bounds__(ConvLaunch<S2, E>::MAXT) split_row(const __grid_constant__ SplitArgs a) {
    using T = cplx<R>;
    using Sh = FftShape<S2, E>;
    constexpr int TT = Sh::T;
    constexpr int NX = MultShape<MULT>::NX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = blockDim.x / TT;
    const int g = threadIdx.x / TT;
    const int tau = threadIdx.x - g * TT;
    T* sm = reinterpret_cast<T*>(smem_raw) + (size_t)g * NX * Sh::SMEM;
    const int64_t row = (int64_t)blockIdx.x * G + g;
    const int64_t rows = a.count * a.nr * (int64_t)a.S1;
    split_row_body<R, S2, E, KIND, MULT>(a, row, row < rows, tau, sm);
}

// Output store of the backward columns: the first residue block stores, the
// later ones add to what the earlier ones stored.
template <class T>
__device__ __forceinline__ void split_store(T* p, T v, int accumulate) {
    if (accumulate) v = cadd(*p, v);
    __stcs(p, v);
}

// Backward column j2 of output b of instance inst; all residues of the block
// accumulated.
template <class R, int S1, int KIND, bool COMP>
__device__ __forceinline__ void split_colbwd_body(const SplitArgs& a, int64_t inst, int b, int j2) {
    using T = cplx<R>;
    constexpr int NB = (KIND == KIND_HERMITIAN) ? 1 : 2;
    const T* twR = static_cast<const T*>(a.twR);
    const T* twS = static_cast<const T*>(a.twS);
    const T* base = static_cast<const T*>(a.work) + (inst * a.P + b) * (int64_t)a.nr * a.S;
    R s0[2 * S1], c0[COMP ? 2 * S1 : 1], s1[NB == 2 ? 2 * S1 : 1], c1[(NB == 2 && COMP) ? 2 * S1 : 1];
    R dummy = 0;
#pragma unroll
    for (int i = 0; i < 2 * S1; ++i) {
        s0[i] = 0;
        if constexpr (COMP) c0[i] = 0;
        if constexpr (NB == 2) {
            s1[i] = 0;
            if constexpr (COMP) c1[i] = 0;
        }
    }
    for (int r = a.r0; r < a.r0 + a.nr; ++r) {
        T cr = ldtw(twR + (int64_t)a.n * a.S + r);
        if constexpr (KIND != KIND_COMPLEX) cr = cconj(cr);
        T v[S1], tw[S1];
        power_row_twiddles<S1, true>(twS + j2, a.S2, tw);   // zeta_S^{j2 k1}
#pragma unroll
        for (int k1 = 0; k1 < S1; ++k1) {
            const T z = base[(int64_t)(r - a.r0) * a.S + (int64_t)k1 * a.S2 + j2];
            v[k1] = k1 == 0 ? z : cmulc(z, tw[k1]);
        }
        dft_small<S1, true>(v);
        const TwistRow tr = twist_row(r, a.n);        // conjugate symmetry
        const T* twr = twR + (int64_t)tr.row * a.S;
        const T tb = twist_ld(twr + j2, tr.conj);     // zeta_N^{r j2}
#pragma unroll
        for (int j1 = 0; j1 < S1; ++j1) {
            T y = cmulc(v[j1], split_twist(twr, tb, j1, a.S2, tr.conj));
            acc_add<R, COMP>(s0[2 * j1], COMP ? c0[2 * j1] : dummy, y.x);
            acc_add<R, COMP>(s0[2 * j1 + 1], COMP ? c0[2 * j1 + 1] : dummy, y.y);
            if constexpr (NB == 2) {
                const T y1 = cmulc(y, cr);
                acc_add<R, COMP>(s1[2 * j1], COMP ? c1[2 * j1] : dummy, y1.x);
                acc_add<R, COMP>(s1[2 * j1 + 1], COMP ? c1[2 * j1 + 1] : dummy, y1.y);
            }
        }
    }
    T* hout = static_cast<T*>(a.h[b]) + inst * a.stride;
    const R sc = R(a.invN);
#pragma unroll
    for (int j1 = 0; j1 < S1; ++j1) {
        const int j = j1 * a.S2 + j2;
        const R x0 = COMP ? s0[2 * j1] + c0[2 * j1] : s0[2 * j1];
        const R y0 = COMP ? s0[2 * j1 + 1] + c0[2 * j1 + 1] : s0[2 * j1 + 1];
        const T o0 = mk<T>(x0 * sc, y0 * sc);
        T o1 = czero<T>();
        if constexpr (NB == 2) {
            const R x1 = COMP ? s1[2 * j1] + c1[2 * j1] : s1[2 * j1];
            const R y1 = COMP ? s1[2 * j1 + 1] + c1[2 * j1 + 1] : s1[2 * j1 + 1];
            o1 = mk<T>(x1 * sc, y1 * sc);
        }
        if constexpr (KIND == KIND_COMPLEX) {
            if (j < a.L) split_store(hout + j, o0, a.accumulate);
            if (j + a.S < a.L) split_store(hout + j + a.S, o1, a.accumulate);
        } else if constexpr (KIND == KIND_CENTERED) {
            if (j < a.L - a.H) split_store(hout + j + a.H, o0, a.accumulate);
            if (j >= a.S - a.H) split_store(hout + j - a.S + a.H, o1, a.accumulate);
        } else {
            if (j < a.Ls) split_store(hout + j, o0, a.accumulate);
        }
    }
}

// U columns j2 = j2base + u * jstep of one instance by one thread, all
// residues: per residue the U * S1 work-buffer loads are issued together.
template <class R, int S1, int KIND, bool COMP, int U>
__device__ __forceinline__ void split_colbwd_multi(const SplitArgs& a, int64_t inst, int j2base, int jstep) {
    using T = cplx<R>;
    constexpr int NB = (KIND == KIND_HERMITIAN) ? 1 : 2;
    constexpr int NA = 2 * S1;
    const T* twR = static_cast<const T*>(a.twR);
    const T* twS = static_cast<const T*>(a.twS);
    const T* base = static_cast<const T*>(a.work) + inst * a.P * (int64_t)a.nr * a.S;   // output 0 (part 0)
    R s0[U][NA], c0[U][COMP ? NA : 1], s1[U][NB == 2 ? NA : 1], c1[U][(NB == 2 && COMP) ? NA : 1];
    R dummy = 0;
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            s0[u][i] = 0;
            if constexpr (COMP) c0[u][i] = 0;
            if constexpr (NB == 2) {
                s1[u][i] = 0;
                if constexpr (COMP) c1[u][i] = 0;
            }
        }
    for (int r = a.r0; r < a.r0 + a.nr; ++r) {
        T cr = ldtw(twR + (int64_t)a.n * a.S + r);
        if constexpr (KIND != KIND_COMPLEX) cr = cconj(cr);
        T v[U][S1];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int k1 = 0; k1 < S1; ++k1)
                v[u][k1] = base[(int64_t)(r - a.r0) * a.S + (int64_t)k1 * a.S2 + j2base + u * jstep];
        const TwistRow tr = twist_row(r, a.n);        // conjugate symmetry
        const T* twr = twR + (int64_t)tr.row * a.S;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j2 = j2base + u * jstep;
            T tw[S1];
            power_row_twiddles<S1, true>(twS + j2, a.S2, tw);   // zeta_S^{j2 k1}
#pragma unroll
            for (int k1 = 1; k1 < S1; ++k1) v[u][k1] = cmulc(v[u][k1], tw[k1]);
            dft_small<S1, true>(v[u]);
            const T tb = twist_ld(twr + j2, tr.conj);  // zeta_N^{r j2}
#pragma unroll
            for (int j1 = 0; j1 < S1; ++j1) {
                T y = cmulc(v[u][j1], split_twist(twr, tb, j1, a.S2, tr.conj));
                acc_add<R, COMP>(s0[u][2 * j1], COMP ? c0[u][2 * j1] : dummy, y.x);
                acc_add<R, COMP>(s0[u][2 * j1 + 1], COMP ? c0[u][2 * j1 + 1] : dummy, y.y);
                if constexpr (NB == 2) {
                    const T y1 = cmulc(y, cr);
                    acc_add<R, COMP>(s1[u][2 * j1], COMP ? c1[u][2 * j1] : dummy, y1.x);
                    acc_add<R, COMP>(s1[u][2 * j1 + 1], COMP ? c1[u][2 * j1 + 1] : dummy, y1.y);
                }
            }
        }
    }
    T* hout = static_cast<T*>(a.h[0]) + inst * a.stride;
    const R sc = R(a.invN);
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int j2 = j2base + u * jstep;
#pragma unroll
        for (int j1 = 0; j1 < S1; ++j1) {
            const int j = j1 * a.S2 + j2;
            const R x0 = COMP ? s0[u][2 * j1] + c0[u][2 * j1] : s0[u][2 * j1];
            const R y0 = COMP ? s0[u][2 * j1 + 1] + c0[u][2 * j1 + 1] : s0[u][2 * j1 + 1];
            const T o0 = mk<T>(x0 * sc, y0 * sc);
            T o1 = czero<T>();
            if constexpr (NB == 2) {
                const R x1 = COMP ? s1[u][2 * j1] + c1[u][2 * j1] : s1[u][2 * j1];
                const R y1 = COMP ? s1[u][2 * j1 + 1] + c1[u][2 * j1 + 1] : s1[u][2 * j1 + 1];
                o1 = mk<T>(x1 * sc, y1 * sc);
            }
            if constexpr (KIND == KIND_COMPLEX) {
                if (j < a.L) split_store(hout + j, o0, a.accumulate);
                if (j + a.S < a.L) split_store(hout + j + a.S, o1, a.accumulate);
            } else if constexpr (KIND == KIND_CENTERED) {
                if (j < a.L - a.H) split_store(hout + j + a.H, o0, a.accumulate);
                if (j >= a.S - a.H) split_store(hout + j - a.S + a.H, o1, a.accumulate);
            } else {
                if (j < a.Ls) split_store(hout + j, o0, a.accumulate);
            }
        }
    }
}

// Backward columns: one thread per (instance, output, j2).
template <class R, int S1, int KIND, bool COMP>
__global__ void __launch_bounds__(256) split_colbwd(const __grid_constant__ SplitArgs a) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= a.count * a.B * (int64_t)a.S2) return;
    const int64_t ib = tid / a.S2;
    split_colbwd_body<R, S1, KIND, COMP>(a, ib / a.B, (int)(ib % a.B), (int)(tid % a.S2));
}

}  // namespace hd
